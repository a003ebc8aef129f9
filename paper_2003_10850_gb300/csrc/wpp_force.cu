// wpp_force.cu -- the default force pass: pairs from the density pass's neighbour
// lists (k_force_list), and the walk for what they cannot serve: member-parallel
// for groups of active particles (k_force_mp), one particle per warp for the rest
// (k_force_wpp).
#include "wpp.cuh"

namespace sph {

// ---------------------------------------------------------------------------
// Force
// ---------------------------------------------------------------------------

// Particle i's Balsara factor and viscosity parameter, and the pair partner's.
template <int VISC>
__device__ __forceinline__ float2 wpp_visc_i(const WppArgs& a, int p) {
    return VISC == kViscPerParticle ? a.fvisc[p] : make_float2(VISC == kViscBalsara ? a.fbal[p] : 1.f, 0.f);
}
template <int VISC>
__device__ __forceinline__ float2 wpp_visc_j(const WppArgs& a, int q) {
    return VISC == kViscPerParticle ? __ldg(a.fvisc + q)
                                    : make_float2(VISC == kViscBalsara ? __ldg(a.fbal + q) : 1.f, 0.f);
}

template <bool HASH, int MINB, int VISC, bool COND>
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
    if (a.fb_act && wpp_lists_valid(a.list_st)) {
        act = a.fb_act;
        cnt = (int)*a.fb_count;
        chunk = 1;
    } else if (a.left) {   // after the member-parallel walk: the particles it left
        act = a.left;
        cnt = (int)*a.left_n;
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
            const WppGroup G = wpp_group(a.boxes, a.n_boxes, act, t, t1, a.grp_shift);
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
                const float2 bi = wpp_visc_i<VISC>(a, p);
                const WppForceI I = {vi.x, vi.y, vi.z, thi.w, thi.x, thi.y, thi.z,
                                     kNorm * thi.w * thi.w * thi.w * thi.w, bi.x, ci.x, ci.y, bi.y};
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
                        wpp_force_pair<VISC, COND>(I, e.x, e.y, e.z, __ldg(a.fvm + q), __ldg(a.fthermo + q),
                                                   wpp_visc_j<VISC>(a, q),
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
                                    if (HHi < 0.0) HHi = wpp_hh(hi, B);
                                    in = exact_pred(D2, HHi);
                                }
                                if (!in && mj) in = exact_pred(D2, wpp_hh(f.w, B));
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

// Force pass from the recorded lists: four active particles per warp, eight
// lanes each, two pairs per lane per step (the neighbour list, then the extra
// partners); the same pair terms as k_force_wpp, folded error-free within
// each octet of lanes. If the lists cannot serve the call at all the kernel
// does nothing and the walk that follows takes the whole active set;
// particles whose own lists did not fit go to fb_list for that walk.
constexpr int kFlPer = 4;   // particles per warp
template <bool HASH, int VISC, bool COND>
__global__ void __launch_bounds__(128, 8) k_force_list(WppArgs a) {
    if (!wpp_lists_valid(a.list_st)) return;
    const unsigned gen = a.list_st[kListGen];
    const unsigned lane = lane_id();
    const int slot = (int)(lane >> 3), sub = (int)(lane & 7u);
    const int warps = gridDim.x * (blockDim.x >> 5);
    const int cnt = (int)*a.count_ptr;
    const float kNorm = (float)(8.0 / 3.141592653589793);
    unsigned long long c_pairs = 0, c_served = 0;   // per octet, lane-uniform within it
    for (int t0 = (blockIdx.x * (blockDim.x >> 5) + (int)(threadIdx.x >> 5)) * kFlPer; t0 < cnt;
         t0 += warps * kFlPer) {
        const int t = t0 + slot;
        int p = -1, cn = 0;
        unsigned ec = 0;
        if (t < cnt) {
            p = a.act[t];
            cn = a.nbr_n[p];
            ec = a.ext_n[p];
            // (kExtUnusable included; a stale stamp: p was not active in the call that recorded)
            if (cn < 0 || ec > (unsigned)kExtCap || a.list_ep[p] != gen) {
                if (sub == 0) a.fb_list[atomicAdd(&a.list_st[3], 1u)] = p;
                p = -1;
            }
        }
        const bool live = p >= 0;
        const int pp = live ? p : 0;
        const BoxDesc& B = a.boxes[a.n_boxes == 1 ? 0 : wpp_box(a.boxes, a.n_boxes, pp)];
        const float sf = B.sf;
        const uint4 Xi = a.posm[pp];
        const int oi = a.perm[pp];
        const float4 vi = a.fvm[pp];
        const float4 thi = a.fthermo[pp];
        const float2 ci = COND ? a.fcond[pp] : make_float2(0.f, 0.f);
        const float2 bi = wpp_visc_i<VISC>(a, pp);
        const WppForceI I = {vi.x, vi.y, vi.z, thi.w, thi.x, thi.y, thi.z, kNorm * thi.w * thi.w * thi.w * thi.w,
                             bi.x, ci.x, ci.y, bi.y};
        float Sx = 0.f, Sy = 0.f, Sz = 0.f, Su = 0.f, Sc = 0.f, vsmax = 0.f;
        unsigned long long hs = 0;
        const int tot = live ? cn + (int)ec : 0;
        const int32_t* ln = a.nbr + (live ? a.nbr_off[pp] : 0);
        const int32_t* le = a.ext + (size_t)pp * kExtCap;
        // two pairs per lane per step (k and k + 8), their loads issued together,
        // and the next step's partner indices loaded ahead of this step's gathers;
        // each lane sums its pairs in the order k, k + 8, k + 16, ...
        auto partner = [&](int k) { return k < cn ? ln[k] : le[k - cn]; };
        int q0n = sub < tot ? partner(sub) : 0;
        int q1n = sub + 8 < tot ? partner(sub + 8) : q0n;
        for (int k = sub; __any_sync(0xffffffffu, k < tot); k += 16) {
            const int q0 = q0n, q1 = q1n;
            if (k + 16 < tot) q0n = partner(k + 16);
            if (k + 24 < tot) q1n = partner(k + 24);
            else q1n = q0n;
            if (k < tot) {
                const int k1 = k + 8;
                const bool two = k1 < tot;
                const uint4 X0 = a.posm[q0], X1 = a.posm[q1];
                const float4 v0 = __ldg(a.fvm + q0), v1 = __ldg(a.fvm + q1);
                const float4 t0v = __ldg(a.fthermo + q0), t1v = __ldg(a.fthermo + q1);
                const float2 b0 = wpp_visc_j<VISC>(a, q0), b1 = wpp_visc_j<VISC>(a, q1);
                const float2 c0 = COND ? __ldg(a.fcond + q0) : make_float2(0.f, 0.f);
                const float2 c1 = COND ? __ldg(a.fcond + q1) : make_float2(0.f, 0.f);
                wpp_force_pair<VISC, COND>(I, (float)(int)(X0.x - Xi.x) * sf, (float)(int)(X0.y - Xi.y) * sf,
                                          (float)(int)(X0.z - Xi.z) * sf, v0, t0v, b0, c0, a.alpha, Sx, Sy, Sz, Su,
                                          Sc, vsmax);
                if (HASH) hs += splitmix64((unsigned long long)a.perm[q0]);
                if (two) {
                    wpp_force_pair<VISC, COND>(I, (float)(int)(X1.x - Xi.x) * sf, (float)(int)(X1.y - Xi.y) * sf,
                                              (float)(int)(X1.z - Xi.z) * sf, v1, t1v, b1, c1, a.alpha, Sx, Sy, Sz,
                                              Su, Sc, vsmax);
                    if (HASH) hs += splitmix64((unsigned long long)a.perm[q1]);
                }
            }
        }
        const float fs = wpp_fold4_oct(Sx, Sy, Sz, Su);
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            vsmax = fmaxf(vsmax, __shfl_xor_sync(0xffffffffu, vsmax, o));
            if (HASH) hs += __shfl_xor_sync(0xffffffffu, hs, o);
        }
        const float cs = COND ? wpp_fold1_oct(Sc) : 0.f;
        if (live) {
            if ((sub & 1) == 0) {
                const int comp = sub >> 1;
                if (comp < 3) a.acc[3 * (size_t)oi + comp] = fs;
                else a.dudt[oi] = fs;
            }
            if (sub == 0) {
                if (COND) a.dudt_cond[oi] = cs;
                a.vsig[oi] = vsmax;
                if (HASH) a.hash[oi] = hs;
                c_pairs += (unsigned long long)tot;
                ++c_served;
            }
        }
    }
    c_pairs = warp_sum(c_pairs);
    c_served = warp_sum(c_served);
    if (lane == 0 && c_pairs) atomicAdd(&a.ctr->force_pairs, c_pairs);
    if (lane == 0 && c_served) atomicAdd(&a.ctr->list_force, c_served);
}


// ---------------------------------------------------------------------------
// Member-parallel force walk (active sets the neighbour lists cannot serve)
// ---------------------------------------------------------------------------
//
// For a group of up to 8 active particles of one leaf-parent node: one walk
// of the hierarchy at radius max(h_max of the group, h_max of the node), then
// one sweep of the group's leaves with one candidate j per lane, decided for
// every member i at once: j is a partner when r_ij < h_i or r_ij < h_j, in
// FP32 outside a thin band around either radius and by the exact predicate
// inside it. Each member's partners go to its pair list in the warp's global
// scratch (kFmCap entries); the pair terms are then summed from the lists, a
// member at a time, as the list-based force pass does. Singletons, groups
// whose leaf list overflows and members whose pair list overflows are left
// to the one-particle walk (k_force_wpp).
constexpr int kFmCap = 256;   // pairs per member in the scratch list
static_assert(kMpMembers * kFmCap <= 2 * kMpMembers * kMpCap, "scratch of a force warp");

struct WppFmSmem {
    int glf[kWppGrpLeaves];
    int stk[kWppStack];
    float4 mem[kMpMembers];   // member offset from the group centre, (h_i (1 + 2^-19) + eb)^2 (1 + 2^-18)
    float lo[kMpMembers];     // (h_i (1 - 2^-19) - eb)^2 (1 - 2^-18): surely inside below this
    float hm[kMpMembers];     // h_i
    uint4 X[kMpMembers];      // integer positions
    int cnt[kMpMembers];      // pairs found per member
    int pm[kMpMembers];       // member sorted indices (-1: no member)
    // candidates that passed the box prefilter, waiting for the member tests:
    // offset from the group centre and h_j (sign bit: a wide leaf's), index
    float4 bp[32];
    int bq[32];
};

template <bool HASH, int MINB, int VISC, bool COND>
__global__ void __launch_bounds__(kWppThreads, MINB) k_force_mp(WppArgs a) {
    // the recorded lists served this call: the walk takes only their fallbacks
    if (a.fb_act && wpp_lists_valid(a.list_st)) return;
    __shared__ WppFmSmem smem[kWppWarps];
    const int wib = (int)(threadIdx.x >> 5);
    WppFmSmem& sm = smem[wib];
    // this warp's pair lists: kMpMembers x kFmCap entries
    int32_t* pj = a.mp_j + ((size_t)blockIdx.x * kWppWarps + wib) * (kMpMembers * kFmCap);
    const unsigned lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    const float rel = 9.5367431640625e-07f;  // 2^-20
    const float elo = 1.f - 4.f * rel, ehi = 1.f + 4.f * rel;
    const float kNorm = (float)(8.0 / 3.141592653589793);
    const int cnt = (int)*a.count_ptr;
    unsigned long long c_pairs = 0, c_tests = 0;   // lane 0
    for (;;) {
        int t0 = 0;
        if (lane == 0) t0 = (int)atomicAdd(a.queue, (unsigned)a.chunk);
        t0 = __shfl_sync(0xffffffffu, t0, 0);
        if (t0 >= cnt) break;
        const int t1 = min(t0 + a.chunk, cnt);
        for (int t = t0; t < t1;) {
            const WppGroup G = wpp_group(a.boxes, a.n_boxes, a.act, t, t1, a.grp_shift);
            t += G.n;
            const BoxDesc& B = a.boxes[G.box];
            const float sf = B.sf;
            const int off = (int)B.off, pend = (int)(B.off + B.n);
            uint4 Xl = make_uint4(0u, 0u, 0u, 0u);
            float hl = 0.f;
            if (G.p >= 0) {
                Xl = a.posm[G.p];
                hl = a.fvel[G.p].w;
            }
            int ngl = -1;
            WppGroupGeom gg;
            if (G.n >= 2 && B.nlev > 1) {
                const float hg = warp_max(hl);
                ngl = wpp_group_leaves(sm, B, a.node_c, a.node_e, Xl, G.p >= 0, sf,
                                       [&](float4 e) { return fmaxf(hg, e.w); }, gg);
            }
            unsigned todo = (1u << G.n) - 1u;   // members left to the one-particle walk
            if (ngl >= 0) {
                const float eT = gg.eb;
                if ((int)lane < kMpMembers) {
                    float4 mem = make_float4(0.f, 0.f, 0.f, -1.f);
                    float lo = -1.f;
                    if ((int)lane < G.n) {
                        const float ti = hl * (1.f + 2.f * rel) + eT, si = fmaxf(hl * (1.f - 2.f * rel) - eT, 0.f);
                        mem = make_float4((float)(int)(Xl.x - gg.Gc.x) * sf, (float)(int)(Xl.y - gg.Gc.y) * sf,
                                          (float)(int)(Xl.z - gg.Gc.z) * sf, ti * ti * ehi);
                        lo = si * si * elo;
                    }
                    sm.mem[lane] = mem;
                    sm.lo[lane] = lo;
                    sm.hm[lane] = hl;
                    sm.X[lane] = Xl;
                    sm.pm[lane] = G.p;   // -1 past G.n
                }
                __syncwarp();
                int cntm[kMpMembers];
#pragma unroll
                for (int k = 0; k < kMpMembers; ++k) cntm[k] = 0;
                // Box prefilter: a candidate goes on to the member tests only if it
                // comes within the largest member threshold, or its own, of the
                // group's box. Both tests run on the same computed offsets; the
                // margin of 2^-12 of the squared radius covers their rounding, so
                // a candidate that some member takes always passes.
                const float Tmax = warp_max((int)lane < kMpMembers ? sm.mem[lane].w : -1.f);
                const float egx = gg.egx, egy = gg.egy, egz = gg.egz;
                unsigned ctest = 0;
                const int lvl0 = B.lvl_off[0];
                auto fetch = [&](int base, int& e, int& q, bool& cand, uint4& C, float4& f) {
                    const int li = base + (int)(lane >> 3);
                    e = li < ngl ? sm.glf[li] : 0;
                    const int qq = off + (e & 0x7fffffff) * kLeaf + (int)(lane & 7u);
                    cand = li < ngl && qq < pend;
                    q = cand ? qq : off;
                    C = a.node_c[lvl0 + (e & 0x7fffffff)];
                    f = __ldg(a.fposh + q);
                };
                // Every member tests the buffer's first kb candidates (one per lane).
                auto members = [&](int kb) {
                    __syncwarp();
                    const bool cand = (int)lane < kb;
                    const float4 f0 = sm.bp[lane];
                    const int q = sm.bq[lane];
                    __syncwarp();   // read before the next candidates overwrite the entry
                    const bool wide = cand && (__float_as_uint(f0.w) >> 31) != 0u;
                    // j side of the band: h_j (1 +- 2^-19) widened/narrowed by the rounding bound
                    const float hj = __uint_as_float(__float_as_uint(f0.w) & 0x7fffffffu);
                    const float tj = hj * (1.f + 2.f * rel) + eT, sj = fmaxf(hj * (1.f - 2.f * rel) - eT, 0.f);
                    const float hij = tj * tj * ehi, loj = sj * sj * elo;
                    const bool anyw = __any_sync(0xffffffffu, wide);
                    uint4 Xq = make_uint4(0u, 0u, 0u, 0u);
                    if (anyw && wide) Xq = a.posm[q];
                    unsigned bandm = 0;   // members for which this lane's pair lies in the band
#pragma unroll
                    for (int m = 0; m < kMpMembers; ++m) {
                        const float4 g = sm.mem[m];
                        float dx = f0.x - g.x, dy = f0.y - g.y, dz = f0.z - g.z;
                        if (anyw) {
                            if (wide) {   // exact integer separations from the member
                                const uint4 Xm = sm.X[m];
                                dx = (float)(int)(Xq.x - Xm.x) * sf;
                                dy = (float)(int)(Xq.y - Xm.y) * sf;
                                dz = (float)(int)(Xq.z - Xm.z) * sf;
                            }
                        }
                        const float r2 = dx * dx + dy * dy + dz * dz;
                        const bool ok = cand && q != sm.pm[m];
                        const bool in = ok && (r2 < sm.lo[m] || r2 < loj);
                        const bool band = ok && !in && (r2 < g.w || r2 < hij);
                        bandm |= band ? 1u << m : 0u;
                        const unsigned msk = __ballot_sync(0xffffffffu, in);
                        const int k = cntm[m] + __popc(msk & lt);
                        if (in && k < kFmCap) pj[m * kFmCap + k] = q;
                        cntm[m] += __popc(msk);
                    }
                    // the rare pairs within the band of either radius: the exact predicate
                    const unsigned anyb = __reduce_or_sync(0xffffffffu, bandm);
                    if (anyb) {
                        const uint4 Xj = (bandm != 0u) ? a.posm[q] : make_uint4(0u, 0u, 0u, 0u);
                        double HHj = -1.0;
#pragma unroll 1
                        for (int m = 0; m < kMpMembers; ++m) {
                            if (!((anyb >> m) & 1u)) continue;
                            bool in = false;
                            if ((bandm >> m) & 1u) {   // r < h_i or r < h_j, exactly
                                const unsigned long long D2 = exact_d2(sm.X[m], Xj);
                                in = exact_pred(D2, wpp_hh(sm.hm[m], B));
                                if (!in) {
                                    if (HHj < 0.0) HHj = wpp_hh(hj, B);
                                    in = exact_pred(D2, HHj);
                                }
                            }
                            const unsigned msk = __ballot_sync(0xffffffffu, in);
                            int c = 0;
#pragma unroll
                            for (int k2 = 0; k2 < kMpMembers; ++k2) c = m == k2 ? cntm[k2] : c;
                            const int k = c + __popc(msk & lt);
                            if (in && k < kFmCap) pj[m * kFmCap + k] = q;
#pragma unroll
                            for (int k2 = 0; k2 < kMpMembers; ++k2) cntm[k2] += m == k2 ? __popc(msk) : 0;
                        }
                    }
                };
                int nb = 0;   // candidates waiting in the buffer (warp-uniform)
                int e_n, q_n;
                bool cand_n;
                uint4 C_n;
                float4 f_n;
                fetch(0, e_n, q_n, cand_n, C_n, f_n);
                for (int base = 0; base < ngl; base += 4) {
                    const int e = e_n, q = q_n;
                    const bool cand = cand_n;
                    const uint4 C = C_n;
                    const float4 f = f_n;
                    if (base + 4 < ngl) fetch(base + 4, e_n, q_n, cand_n, C_n, f_n);
                    const float px = (float)(int)(C.x - gg.Gc.x) * sf + f.x, py = (float)(int)(C.y - gg.Gc.y) * sf + f.y,
                                pz = (float)(int)(C.z - gg.Gc.z) * sf + f.z;
                    const bool wide = cand && e < 0;
                    ctest += __popc(__ballot_sync(0xffffffffu, cand));
                    // a wide leaf's offsets are not accurate enough for the box test: it passes
                    bool pass = cand;
                    if (cand && !wide) {
                        const float bx = fmaxf(fabsf(px) - egx, 0.f), by = fmaxf(fabsf(py) - egy, 0.f),
                                    bz = fmaxf(fabsf(pz) - egz, 0.f);
                        const float tj = f.w * (1.f + 2.f * rel) + eT;
                        const float T = fmaxf(Tmax, tj * tj * ehi) * (1.f + 2.44140625e-4f);
                        pass = bx * bx + by * by + bz * bz < T;
                    }
                    const unsigned pb = __ballot_sync(0xffffffffu, pass);
                    const int slot = nb + __popc(pb & lt);
                    const float4 ent = make_float4(px, py, pz,
                                                   __uint_as_float(__float_as_uint(f.w) | (wide ? 0x80000000u : 0u)));
                    if (pass && slot < 32) {
                        sm.bp[slot] = ent;
                        sm.bq[slot] = q;
                    }
                    nb += __popc(pb);
                    if (nb >= 32) {
                        members(32);
                        if (pass && slot >= 32) {
                            sm.bp[slot - 32] = ent;
                            sm.bq[slot - 32] = q;
                        }
                        nb -= 32;
                    }
                }
                if (nb > 0) members(nb);
                if (lane == 0) c_tests += (unsigned long long)ctest * (unsigned)G.n;
                // members whose list overflowed go to the one-particle walk
                todo = 0;
                int cmine = 0;
#pragma unroll
                for (int k = 0; k < kMpMembers; ++k) {
                    todo |= (k < G.n && cntm[k] > kFmCap) ? 1u << k : 0u;
                    cmine = (int)lane == k ? cntm[k] : cmine;
                }
                if ((int)lane < kMpMembers) sm.cnt[lane] = cmine;
                __syncwarp();
                // pair terms from the members' lists as k_force_list sums them: four
                // members at a time, eight lanes each, two pairs per lane per step with
                // the next step's partner indices loaded ahead
                for (int m0 = 0; m0 < G.n; m0 += 4) {
                    const int m = m0 + (int)(lane >> 3), sub = (int)(lane & 7u);
                    const int tot0 = m < G.n ? sm.cnt[m] : 0;
                    const bool live = m < G.n && tot0 <= kFmCap;
                    const int tot = live ? tot0 : 0;
                    const int mq = m < G.n ? m : 0;
                    const int p = __shfl_sync(0xffffffffu, G.p, mq);
                    const uint4 Xi = sm.X[mq];
                    const int oi = a.perm[p];
                    const float4 vi = a.fvm[p];
                    const float4 thi = a.fthermo[p];
                    const float2 ci = COND ? a.fcond[p] : make_float2(0.f, 0.f);
                    const float2 bi = wpp_visc_i<VISC>(a, p);
                    const WppForceI I = {vi.x, vi.y, vi.z, thi.w, thi.x, thi.y, thi.z,
                                         kNorm * thi.w * thi.w * thi.w * thi.w, bi.x, ci.x, ci.y, bi.y};
                    float Sx = 0.f, Sy = 0.f, Sz = 0.f, Su = 0.f, Sc = 0.f, vsmax = 0.f;
                    unsigned long long hs = 0;
                    const int32_t* lst = pj + mq * kFmCap;
                    int q0n = sub < tot ? lst[sub] : 0;
                    int q1n = sub + 8 < tot ? lst[sub + 8] : q0n;
                    for (int k = sub; __any_sync(0xffffffffu, k < tot); k += 16) {
                        const int q0 = q0n, q1 = q1n;
                        if (k + 16 < tot) q0n = lst[k + 16];
                        q1n = k + 24 < tot ? lst[k + 24] : q0n;
                        if (k < tot) {
                            const bool two = k + 8 < tot;
                            const uint4 X0 = a.posm[q0], X1 = a.posm[q1];
                            const float4 v0 = __ldg(a.fvm + q0), v1 = __ldg(a.fvm + q1);
                            const float4 th0 = __ldg(a.fthermo + q0), th1 = __ldg(a.fthermo + q1);
                            const float2 b0 = wpp_visc_j<VISC>(a, q0), b1 = wpp_visc_j<VISC>(a, q1);
                            const float2 c0 = COND ? __ldg(a.fcond + q0) : make_float2(0.f, 0.f);
                            const float2 c1 = COND ? __ldg(a.fcond + q1) : make_float2(0.f, 0.f);
                            wpp_force_pair<VISC, COND>(I, (float)(int)(X0.x - Xi.x) * sf,
                                                       (float)(int)(X0.y - Xi.y) * sf, (float)(int)(X0.z - Xi.z) * sf,
                                                       v0, th0, b0, c0, a.alpha, Sx, Sy, Sz, Su, Sc, vsmax);
                            if (HASH) hs += splitmix64((unsigned long long)a.perm[q0]);
                            if (two) {
                                wpp_force_pair<VISC, COND>(I, (float)(int)(X1.x - Xi.x) * sf,
                                                           (float)(int)(X1.y - Xi.y) * sf,
                                                           (float)(int)(X1.z - Xi.z) * sf, v1, th1, b1, c1, a.alpha,
                                                           Sx, Sy, Sz, Su, Sc, vsmax);
                                if (HASH) hs += splitmix64((unsigned long long)a.perm[q1]);
                            }
                        }
                    }
                    const float fs = wpp_fold4_oct(Sx, Sy, Sz, Su);
#pragma unroll
                    for (int o = 4; o > 0; o >>= 1) {
                        vsmax = fmaxf(vsmax, __shfl_xor_sync(0xffffffffu, vsmax, o));
                        if (HASH) hs += __shfl_xor_sync(0xffffffffu, hs, o);
                    }
                    const float cs = COND ? wpp_fold1_oct(Sc) : 0.f;
                    if (live) {
                        if ((sub & 1) == 0) {
                            const int comp = sub >> 1;
                            if (comp < 3) a.acc[3 * (size_t)oi + comp] = fs;
                            else a.dudt[oi] = fs;
                        }
                        if (sub == 0) {
                            if (COND) a.dudt_cond[oi] = cs;
                            a.vsig[oi] = vsmax;
                            if (HASH) a.hash[oi] = hs;
                        }
                    }
                    // lane 0 keeps the warp's pair count
                    const int tsum = __shfl_sync(0xffffffffu, tot, 0) + __shfl_sync(0xffffffffu, tot, 8) +
                                     __shfl_sync(0xffffffffu, tot, 16) + __shfl_sync(0xffffffffu, tot, 24);
                    if (lane == 0) c_pairs += (unsigned long long)tsum;
                }
                __syncwarp();
            }
            // the members left over go to the one-particle walk
            if (todo) {
                unsigned o = 0;
                if (lane == 0) o = atomicAdd(a.left_n, (unsigned)__popc(todo));
                o = __shfl_sync(0xffffffffu, o, 0);
                if ((int)lane < G.n && ((todo >> lane) & 1u)) a.left[o + __popc(todo & lt)] = G.p;
            }
        }
    }
    if (lane == 0) {
        atomicAdd(&a.ctr->force_pairs, c_pairs);
        atomicAdd(&a.ctr->pair_tests, c_tests);
    }
}

// Kernel variants of the force pass: hash output, register budget,
// viscosity (kViscScalar ...), conduction. Per-particle viscosity comes
// without conduction (no entry point asks for both).
template <bool H, int V, bool C>
static void launch_fl(int blocks, cudaStream_t s, const WppArgs& c) {
    k_force_list<H, V, C><<<blocks, 128, 0, s>>>(c);
}
template <bool H>
static void launch_fl_v(int visc, bool cond, int blocks, cudaStream_t s, const WppArgs& c) {
    if (visc == kViscPerParticle) launch_fl<H, kViscPerParticle, false>(blocks, s, c);
    else if (visc == kViscBalsara) cond ? launch_fl<H, kViscBalsara, true>(blocks, s, c)
                                        : launch_fl<H, kViscBalsara, false>(blocks, s, c);
    else cond ? launch_fl<H, kViscScalar, true>(blocks, s, c) : launch_fl<H, kViscScalar, false>(blocks, s, c);
}
static void launch_force_list(bool hash, int visc, bool cond, int blocks, cudaStream_t s, const WppArgs& c) {
    hash ? launch_fl_v<true>(visc, cond, blocks, s, c) : launch_fl_v<false>(visc, cond, blocks, s, c);
}
template <bool H, int M>
static void launch_fw(int visc, bool cond, int blocks, cudaStream_t s, const WppArgs& c) {
    if (visc == kViscPerParticle) k_force_wpp<H, M, kViscPerParticle, false><<<blocks, kWppThreads, 0, s>>>(c);
    else if (visc == kViscBalsara) {
        if (cond) k_force_wpp<H, M, kViscBalsara, true><<<blocks, kWppThreads, 0, s>>>(c);
        else k_force_wpp<H, M, kViscBalsara, false><<<blocks, kWppThreads, 0, s>>>(c);
    } else {
        if (cond) k_force_wpp<H, M, kViscScalar, true><<<blocks, kWppThreads, 0, s>>>(c);
        else k_force_wpp<H, M, kViscScalar, false><<<blocks, kWppThreads, 0, s>>>(c);
    }
}
template <bool H>
static void launch_fm(int visc, bool cond, int blocks, cudaStream_t s, const WppArgs& c) {
    constexpr int M = kWppFmBps;
    if (visc == kViscPerParticle) k_force_mp<H, M, kViscPerParticle, false><<<blocks, kWppThreads, 0, s>>>(c);
    else if (visc == kViscBalsara) {
        if (cond) k_force_mp<H, M, kViscBalsara, true><<<blocks, kWppThreads, 0, s>>>(c);
        else k_force_mp<H, M, kViscBalsara, false><<<blocks, kWppThreads, 0, s>>>(c);
    } else {
        if (cond) k_force_mp<H, M, kViscScalar, true><<<blocks, kWppThreads, 0, s>>>(c);
        else k_force_mp<H, M, kViscScalar, false><<<blocks, kWppThreads, 0, s>>>(c);
    }
}
static void launch_force_walk(bool hash, bool six, int visc, bool cond, int blocks, cudaStream_t s,
                              const WppArgs& c) {
    if (six) hash ? launch_fw<true, 6>(visc, cond, blocks, s, c) : launch_fw<false, 6>(visc, cond, blocks, s, c);
    else hash ? launch_fw<true, 8>(visc, cond, blocks, s, c) : launch_fw<false, 8>(visc, cond, blocks, s, c);
}

cudaError_t launch_force_wpp(sph_ctx* ctx, const ForceLaunch& a, int64_t n_active, cudaStream_t s) {
    sph_grid* g = const_cast<sph_grid*>(a.g);
    cudaError_t e;
    const bool lists = g->nbr != nullptr && g->lists_rec;
    if (lists && (e = cudaMemsetAsync(g->list_st + 2, 0, 2 * sizeof(unsigned), s))) return e;
    force_pack(g, a.vel, a.u, a.h, a.rho, a.omega, (float)a.gamma, s, lists ? g->list_xh : nullptr,
               lists ? g->list_st + 2 : nullptr, a.divv, a.curlv, a.kappa, a.alpha_v);
    ++ctx->launches;
    if ((e = cudaMemsetAsync(ctx->queue + 3, 0, sizeof(unsigned), s))) return e;
    WppArgs c = wpp_common(ctx, g, ctx->queue + 3);
    c.grp_shift = wpp_grp_shift(a.group_span);
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
    const int visc = a.alpha_v ? kViscPerParticle : a.divv ? kViscBalsara : kViscScalar;
    c.fbal = visc == kViscBalsara ? g->fbal : nullptr;
    c.fvisc = visc == kViscPerParticle ? g->fvisc : nullptr;
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
        c.ext_n = g->ext_n;
        c.list_st = g->list_st;
        c.list_ep = g->list_ep;
        c.fb_list = g->fb_list;
        const int lb = (int)std::max<long long>(
            1, std::min<long long>((long long)ctx->sm_count * 16, (n_active + 4 * kFlPer - 1) / (4 * kFlPer)));
        launch_force_list(a.hash != nullptr, visc, c.fcond != nullptr, lb, s, c);
        ++ctx->launches;
        c.fb_act = g->fb_list;
        c.fb_count = g->list_st + 3;
    }
    // the walk: member-parallel for groups (nothing to do when the lists served
    // the call), then one particle per warp for what it leaves and for the
    // particles the lists could not serve
    if (g->ctx->sm_count >= ctx->sm_count && wpp_groups_pay(ctx, n_active, g->n)) {
        if ((e = cudaMemsetAsync(ctx->queue + 6, 0, 2 * sizeof(unsigned), s))) return e;
        WppArgs cm = c;
        cm.mp_j = g->mp_j;
        cm.left = g->den_left;
        cm.left_n = ctx->queue + 6;
        cm.chunk = kMpMembers;   // whole groups per queue grab
        // a force warp uses the scratch of two density warps: at most half as many warps
        const int fb = std::min(blocks, ctx->sm_count * (kMpWarpsPerSm / (2 * kWppWarps)));
        a.hash ? launch_fm<true>(visc, c.fcond != nullptr, fb, s, cm)
               : launch_fm<false>(visc, c.fcond != nullptr, fb, s, cm);
        ++ctx->launches;
        c.left = g->den_left;
        c.left_n = ctx->queue + 6;
        c.queue = ctx->queue + 7;
    }
    launch_force_walk(a.hash != nullptr, bps <= 6, visc, c.fcond != nullptr, blocks, s, c);
    ++ctx->launches;
    if ((e = span_end(ctx, sp, s))) return e;
    return cudaGetLastError();
}

}  // namespace sph
