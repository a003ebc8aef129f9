// wpp_density.cu -- the default density pass (k_density_mp for groups of active
// particles that share one walk, k_density_wpp one particle per warp for the
// particles it leaves and for sparse active sets) and the neighbour-list build
// that lets the force pass reuse its pair sets (k_list_ext, k_list_sort).
#include "wpp.cuh"

namespace sph {

// ---------------------------------------------------------------------------
// Density
// ---------------------------------------------------------------------------

// Member-parallel path of the density pass (groups of >= 2 members that have a
// group leaf list; at full activity a group is one leaf of 8 particles):
// - candidates: the group's leaf list is swept once, one candidate per lane
//   (lanes 8k..8k+7 on one leaf), each candidate load tested against every
//   member; the pairs within a member's walk radius go to that member's near
//   list in shared memory ((r^2, m)) and global scratch (the index);
// - h iteration: lanes 4m..4m+3 serve member m, each summing every fourth
//   entry of its near list; the four partial sums are folded error-free and
//   the safeguarded Newton step runs for all members at once;
// - a last sweep at the final h records the neighbour lists (and sums the
//   velocity divergence and curl, and the set checksums).
// A member whose near list overflows or whose h leaves its walk radius takes
// the whole-warp path of one particle afterwards.
constexpr int kMpStride = kMpCap + 4;   // float2 entries per member row: rows start 32 bytes apart mod 128
struct WppMpSmem {
    float2 d[kMpMembers][kMpStride];    // (r^2, m_j) of each member's near list
    float4 mem[kMpMembers];             // member offset from the group centre (box units), inclusive threshold
    uint4 X[kMpMembers];                // member integer positions (and mass bits)
    int pm[kMpMembers];                 // member sorted indices (-1: no member)
    // candidates that passed the box prefilter, waiting for the member tests:
    // offset from the group centre and mass (sign bit: a wide leaf's), index,
    // and (partial calls) the inactive candidate's squared reach (-1: active)
    float4 bp[32];
    int bq[32];
    float bt[32];
};
constexpr int kGlfBytes = (int)sizeof(int) * kWppGrpLeaves;   // WppSmem starts with glf
constexpr int kDenSmemWarp = (int)(sizeof(WppSmem) > kGlfBytes + sizeof(WppMpSmem) ? sizeof(WppSmem)
                                                                                      : kGlfBytes + sizeof(WppMpSmem));
static_assert(kWppWarps * kDenSmemWarp <= 48 * 1024, "static shared memory of the density block");
// five resident blocks per SM (the 96-register budget) must fit the SM's 228 KB,
// with the 1 KB the hardware reserves per block
static_assert(5 * (kWppWarps * kDenSmemWarp + 1024) <= 228 * 1024, "five density blocks per SM");

// Error-free (TwoSum) fold of two per-lane sums over aligned quads of lanes:
// every lane of the quad ends with both totals as (s, c), value s - c.
__device__ __forceinline__ void wpp_fold_quad2(float& s1, float& c1, float& s2, float& c2) {
    auto two_sum = [](float& s, float& c, float s2_, float c2_) {
        const float t = __fadd_rn(s, s2_);
        const float bp = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(s2_, bp));
        s = t;
        c = __fsub_rn(__fadd_rn(c, c2_), e);
    };
    c1 = 0.f;
    c2 = 0.f;
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
        const float a1 = __shfl_xor_sync(0xffffffffu, s1, o), b1 = __shfl_xor_sync(0xffffffffu, c1, o);
        const float a2 = __shfl_xor_sync(0xffffffffu, s2, o), b2 = __shfl_xor_sync(0xffffffffu, c2, o);
        two_sum(s1, c1, a1, b1);
        two_sum(s2, c2, a2, b2);
    }
}

// PART: a call on part of the particles that records lists; each member also
// collects its extra partners among the inactive particles (j with
// h_i <= r_ij < h_j), whose h is fixed: the walk reaches the inactive
// particles' h_max (node_e.w, refreshed for this call), and the sweep keeps
// inactive candidates within h_j beyond the member's near radius in a "far"
// list in the warp's scratch.
template <bool HASH, int MINB, bool DIVCURL, bool PART>
__global__ void __launch_bounds__(kWppThreads, MINB) k_density_mp(WppArgs a) {
    __shared__ __align__(16) unsigned char sraw[kWppWarps][kDenSmemWarp];
    const int wib = (int)(threadIdx.x >> 5);
    WppSmem& sm = *reinterpret_cast<WppSmem*>(sraw[wib]);
    WppMpSmem& mp = *reinterpret_cast<WppMpSmem*>(sraw[wib] + kGlfBytes);
    int32_t* mpj = a.mp_j ? a.mp_j + ((size_t)blockIdx.x * kWppWarps + wib) * (kMpMembers * kMpCap) : nullptr;
    int32_t* mpx = PART ? a.mp_x + ((size_t)blockIdx.x * kWppWarps + wib) * (kMpMembers * kMpFar) : nullptr;
    const unsigned gen = a.list_st ? a.list_st[kListGen] : 0u;   // this call's generation
    const unsigned lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    const float rel = 9.5367431640625e-07f;  // 2^-20
    const float nt = (float)a.n_target, nt3 = 3.f * nt, tol3 = 3.f * (float)a.n_tol;
    const int cnt = (int)*a.count_ptr;
    // per-lane counters, summed over the warp at the end
    unsigned c_pairs = 0, c_evals = 0, c_status = 0, c_lists = 0;
    unsigned long long c_tests = 0;
    long long ch_next = 0, ch_end = 0;   // the warp's current chunk of the neighbour-list pool
    // Space for n list entries from the warp's chunk of the pool (warp-uniform
    // n); returns the first entry, or -1 if the pool is full.
    auto reserve = [&](int n) -> long long {
        if (n > a.list_chunk) {
            unsigned long long o = 0;
            if (lane == 0) o = atomicAdd(reinterpret_cast<unsigned long long*>(a.list_st + 4), (unsigned long long)n);
            o = __shfl_sync(0xffffffffu, o, 0);
            return (long long)o + n <= a.list_pool ? (long long)o : -1;
        }
        if (ch_next + n > ch_end) {
            unsigned long long o = 0;
            if (lane == 0)
                o = atomicAdd(reinterpret_cast<unsigned long long*>(a.list_st + 4), (unsigned long long)a.list_chunk);
            o = __shfl_sync(0xffffffffu, o, 0);
            ch_next = (long long)o;
            ch_end = ch_next + a.list_chunk;
        }
        const long long r = ch_next + n <= a.list_pool ? ch_next : -1;
        ch_next += n;
        return r;
    };
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
            float Rg = 0.f;
            WppGroupGeom gg;
            if (G.n >= 2 && B.nlev > 1) {
                Rg = warp_max(a.fixed_h ? hl : hl * a.walk_r);
                ngl = wpp_group_leaves(sm, B, a.node_c, a.node_e, Xl, G.p >= 0, sf,
                                       [&](float4 e) { return PART ? fmaxf(Rg, e.w) : Rg; }, gg);
            }
            unsigned todo = (1u << G.n) - 1u;   // members left for the one-particle path
            if (ngl >= 0 && mpj && G.n >= 2) {
                // ---------------- candidates: one sweep of the group's leaves ----------------
                // 32 candidates per step (the next step's loaded while this one's are
                // tested); those within reach of the group's box wait in a buffer,
                // and every 32 of them go through the member tests.
                const float eT = gg.eb;   // rounding bound of a computed separation (non-wide leaves)
                if ((int)lane < kMpMembers) {
                    float4 mem = make_float4(0.f, 0.f, 0.f, -1.f);
                    if ((int)lane < G.n) {
                        const float Rw = a.fixed_h ? hl : hl * a.walk_r;
                        const float tR = Rw + eT + 2.f * rel * Rw;
                        mem = make_float4((float)(int)(Xl.x - gg.Gc.x) * sf, (float)(int)(Xl.y - gg.Gc.y) * sf,
                                          (float)(int)(Xl.z - gg.Gc.z) * sf, tR * tR * (1.f + 4.f * rel));
                    }
                    mp.mem[lane] = mem;
                    mp.X[lane] = Xl;
                    mp.pm[lane] = G.p;   // -1 past G.n
                }
                __syncwarp();
                int cntm[kMpMembers];
#pragma unroll
                for (int k = 0; k < kMpMembers; ++k) cntm[k] = 0;
                // Box prefilter: a candidate goes on to the member tests only if it
                // comes within the largest member threshold of the group's box (or,
                // PART, within its own h of it). Both tests run on the same computed
                // offsets; the margin of 2^-12 of the squared radius covers their
                // rounding, so a candidate that some member takes always passes.
                const float Tmax = warp_max((int)lane < kMpMembers ? mp.mem[lane].w : -1.f) * (1.f + 2.44140625e-4f);
                const float egx = gg.egx, egy = gg.egy, egz = gg.egz;
                unsigned ctest = 0;
                const int lvl0 = B.lvl_off[0];
                // the candidate of this lane in step `base`: leaf entry, index, centre, (offset, mass)
                auto fetch = [&](int base, int& e, int& q, bool& cand, uint4& C, float4& f) {
                    const int li = base + (int)(lane >> 3);
                    e = li < ngl ? sm.glf[li] : 0;
                    const int qq = off + (e & 0x7fffffff) * kLeaf + (int)(lane & 7u);
                    cand = li < ngl && qq < pend;
                    q = cand ? qq : off;
                    C = a.node_c[lvl0 + (e & 0x7fffffff)];
                    f = __ldg(a.posf + q);
                };
                // Every member tests the buffer's first kb candidates (one per lane)
                // without a branch (a member slot past G.n has a negative
                // threshold), so the eight members' dependent chains interleave.
                auto members = [&](int kb) {
                    __syncwarp();
                    const bool cand = (int)lane < kb;
                    const float4 f0 = mp.bp[lane];
                    const int q = mp.bq[lane];
                    const float Tj = PART ? mp.bt[lane] : -1.f;
                    __syncwarp();   // read before the next candidates overwrite the entry
                    const bool wide = cand && (__float_as_uint(f0.w) >> 31) != 0u;
                    const float mj = __uint_as_float(__float_as_uint(f0.w) & 0x7fffffffu);
                    const bool ina = PART && cand && Tj >= 0.f;
                    const bool anyina = PART && __any_sync(0xffffffffu, ina);
                    if (!__any_sync(0xffffffffu, wide)) {
#pragma unroll
                        for (int m = 0; m < kMpMembers; ++m) {
                            const float4 g = mp.mem[m];
                            const float dx = f0.x - g.x, dy = f0.y - g.y, dz = f0.z - g.z;
                            const float r2 = dx * dx + dy * dy + dz * dz;
                            const bool in = cand && q != mp.pm[m] && r2 < g.w;
                            const unsigned msk = __ballot_sync(0xffffffffu, in);
                            const int k = (cntm[m] & 0xffff) + __popc(msk & lt);
                            if (in && k < kMpCap) {
                                mp.d[m][k] = make_float2(r2, mj);
                                mpj[m * kMpCap + k] = q;
                            }
                            cntm[m] += __popc(msk);
                            if (anyina) {
                                const bool far = ina && m < G.n && !(r2 < g.w) && r2 < Tj;
                                const unsigned fm = __ballot_sync(0xffffffffu, far);
                                const int kf = (cntm[m] >> 16) + __popc(fm & lt);
                                if (far && kf < kMpFar) mpx[m * kMpFar + kf] = q;
                                cntm[m] += __popc(fm) << 16;
                            }
                        }
                    } else {
                        // a wide leaf among them: exact integer separations from each member there
                        const uint4 Xq = wide ? a.posm[q] : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                        for (int m = 0; m < kMpMembers; ++m) {
                            const float4 g = mp.mem[m];
                            float dx = f0.x - g.x, dy = f0.y - g.y, dz = f0.z - g.z;
                            if (wide) {
                                const uint4 Xm = mp.X[m];
                                dx = (float)(int)(Xq.x - Xm.x) * sf;
                                dy = (float)(int)(Xq.y - Xm.y) * sf;
                                dz = (float)(int)(Xq.z - Xm.z) * sf;
                            }
                            const float r2 = dx * dx + dy * dy + dz * dz;
                            const bool in = cand && q != mp.pm[m] && r2 < g.w;
                            const unsigned msk = __ballot_sync(0xffffffffu, in);
                            const int k = (cntm[m] & 0xffff) + __popc(msk & lt);
                            if (in && k < kMpCap) {
                                mp.d[m][k] = make_float2(r2, mj);
                                mpj[m * kMpCap + k] = q;
                            }
                            cntm[m] += __popc(msk);
                            if (anyina) {
                                const bool far = ina && m < G.n && !(r2 < g.w) && r2 < Tj;
                                const unsigned fm = __ballot_sync(0xffffffffu, far);
                                const int kf = (cntm[m] >> 16) + __popc(fm & lt);
                                if (far && kf < kMpFar) mpx[m * kMpFar + kf] = q;
                                cntm[m] += __popc(fm) << 16;
                            }
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
                    // PART: candidate j inactive, and the square of its h widened by the
                    // rounding bound (the far test is inclusive; the last sweep decides)
                    float Tj = -1.f;
                    if (PART && cand && a.flagp[q] == 0) {
                        const float tj = __uint_as_float(a.list_xh[q].w) * (1.f + 2.f * rel) + eT;
                        Tj = tj * tj * (1.f + 4.f * rel);
                    }
                    const float px = (float)(int)(C.x - gg.Gc.x) * sf + f.x, py = (float)(int)(C.y - gg.Gc.y) * sf + f.y,
                                pz = (float)(int)(C.z - gg.Gc.z) * sf + f.z;
                    const bool wide = cand && e < 0;
                    ctest += __popc(__ballot_sync(0xffffffffu, cand));
                    // a wide leaf's offsets are not accurate enough for the box test: it passes
                    bool pass = cand;
                    if (cand && !wide) {
                        const float bx = fmaxf(fabsf(px) - egx, 0.f), by = fmaxf(fabsf(py) - egy, 0.f),
                                    bz = fmaxf(fabsf(pz) - egz, 0.f);
                        const float b2 = bx * bx + by * by + bz * bz;
                        pass = b2 < Tmax || (PART && b2 < Tj * (1.f + 2.44140625e-4f));
                    }
                    const unsigned pb = __ballot_sync(0xffffffffu, pass);
                    const int slot = nb + __popc(pb & lt);
                    const float4 ent = make_float4(px, py, pz,
                                                   __uint_as_float(__float_as_uint(f.w) | (wide ? 0x80000000u : 0u)));
                    if (pass && slot < 32) {
                        mp.bp[slot] = ent;
                        mp.bq[slot] = q;
                        if (PART) mp.bt[slot] = Tj;
                    }
                    nb += __popc(pb);
                    if (nb >= 32) {
                        members(32);
                        if (pass && slot >= 32) {
                            mp.bp[slot - 32] = ent;
                            mp.bq[slot - 32] = q;
                            if (PART) mp.bt[slot - 32] = Tj;
                        }
                        nb -= 32;
                    }
                }
                if (nb > 0) members(nb);
                if (lane == 0) c_tests += (unsigned long long)ctest * (unsigned)G.n;
                __syncwarp();
                // ---------------- h iteration: lanes 4m..4m+3 serve member m ----------------
                const int mm = (int)(lane >> 2), sub = (int)(lane & 3u);
                int cm = 0;
#pragma unroll
                for (int k = 0; k < kMpMembers; ++k) cm = mm == k ? cntm[k] : cm;
                const int cf = PART ? (cm >> 16) : 0;   // far entries (inactive, beyond the near radius)
                cm &= 0xffff;
                const bool mval = mm < G.n;
                float h = __shfl_sync(0xffffffffu, hl, mm);
                const int pm = __shfl_sync(0xffffffffu, G.p, mm);
                const int oim = __shfl_sync(0xffffffffu, ol, mm);
                const uint4 Xm = mp.X[mm];
                const int32_t* jm = mpj + mm * kMpCap;
                const float Rwm = a.fixed_h ? h : h * a.walk_r;
                bool run = mval && cm <= kMpCap;
                bool rew = mval && cm > kMpCap;   // near list overflowed: one-particle path
                float blo = 0.f, bhi = INFINITY, dold = INFINITY;
                unsigned st = 0;
                float fSmw = 0.f, fSmdw = 0.f;   // the final evaluation's per-lane mass sums
                int fnn = 0;
                for (int it = 0;; ++it) {
                    if (!__any_sync(0xffffffffu, run)) break;
                    const float hinv = 1.f / h;
                    const float eL = eT + 2.f * rel * h;
                    const float hi2 = (h + eL) * (h + eL) * (1.f + 4.f * rel);
                    const float lo2 = h > eL ? (h - eL) * (h - eL) * (1.f - 4.f * rel) : 0.f;
                    double HH = -1.0;
                    const bool self = run && sub == 0;   // the self term: w(0) = 1, q w'(0) = 0
                    float Sw = self ? 1.f : 0.f, Sdw = 0.f, Smw = self ? __uint_as_float(Xm.w) : 0.f, Smdw = 0.f;
                    int nn = 0;
                    const int kend = run ? cm : 0;
                    // two entries per lane per step (k and k + 4), independent until the sums
                    auto take = [&](int k) {
                        const float2 e = mp.d[mm][k];
                        bool in = e.x < lo2;
                        if (!in && e.x < hi2) {   // the thin band: the exact predicate
                            if (HH < 0.0) HH = wpp_hh(h, B);
                            in = exact_pred(exact_d2(Xm, a.posm[jm[k]]), HH);
                        }
                        return in ? e : make_float2(-1.f, 0.f);
                    };
                    auto term = [&](float2 e) {
                        if (e.x < 0.f) return;
                        const float qq = (e.x > 0.f ? e.x * rsqrtf(e.x) : 0.f) * hinv;
                        float w, dw;
                        spline<float>(qq, w, dw);
                        const float qdw = qq * dw;
                        Sw += w;
                        Sdw += qdw;
                        Smw += e.y * w;
                        Smdw += e.y * qdw;
                        ++nn;
                    };
                    for (int k = sub; __any_sync(0xffffffffu, k < kend); k += 8) {
                        const float2 e0 = k < kend ? take(k) : make_float2(-1.f, 0.f);
                        const float2 e1 = k + 4 < kend ? take(k + 4) : make_float2(-1.f, 0.f);
                        term(e0);
                        term(e1);
                    }
                    float Cw, Cdw;
                    wpp_fold_quad2(Sw, Cw, Sdw, Cdw);
                    if (run) {
                        if (sub == 0) ++c_evals;
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
                        if (done) {
                            run = false;
                            fSmw = Smw;
                            fSmdw = Smdw;
                            fnn = nn;
                        } else if (!(h <= Rwm * 0.99999f)) {
                            run = false;   // h left the walk radius: one-particle path from this h
                            rew = true;
                        }
                    }
                }
                // ---------------- final: outputs, lists, div/curl, checksums ----------------
                const bool okm = mval && !rew;
                float Cmw, Cmdw;
                wpp_fold_quad2(fSmw, Cmw, fSmdw, Cmdw);
                int nnm = fnn + __shfl_xor_sync(0xffffffffu, fnn, 1);
                nnm += __shfl_xor_sync(0xffffffffu, nnm, 2);
                if (!okm) nnm = 0;
                long long loff = -1;
                if (a.nbr) {
                    int pre = 0, tot = 0;
#pragma unroll
                    for (int k = 0; k < kMpMembers; ++k) {
                        const int v = __shfl_sync(0xffffffffu, nnm, 4 * k);
                        pre += k < mm ? v : 0;
                        tot += v;
                    }
                    const long long gb = tot > 0 ? reserve(tot) : 0;   // (empty lists need no space)
                    loff = gb >= 0 ? gb + pre : -1;
                }
                const bool rec = loff >= 0 && nnm > 0;
                // PART: member mm's extra partners among the inactive particles go
                // straight into its segment (the transpose adds the active ones after)
                int nex = 0;
                int32_t* seg = PART && pm >= 0 ? a.ext + (size_t)pm * kExtCap : nullptr;
                auto add_extra = [&](bool xt, int q) {
                    const unsigned xb = (__ballot_sync(0xffffffffu, xt) >> (4 * mm)) & 0xfu;
                    const int sl = nex + __popc(xb & ((1u << sub) - 1u));
                    if (xt && sl < kExtCap) seg[sl] = q;
                    nex += __popc(xb);
                };
                // r_ij < h_j for a partner with position and h bits Xq: FP32 outside a
                // band of 2^-20 around h_j^2 (integer units), the exact predicate inside
                auto within_hj = [&](uint4 Xq) {
                    const float hj = __uint_as_float(Xq.w);
                    const unsigned long long D2 = exact_d2(Xm, Xq);
                    const float d2 = __ull2float_rn(D2), Hj = hj * B.Hs, H2 = Hj * Hj;
                    if (d2 < H2 * (1.f - rel)) return true;
                    if (d2 > H2 * (1.f + rel)) return false;
                    return exact_pred(D2, wpp_hh(hj, B));
                };
                unsigned long long hs = 0;
                float Dd = 0.f, Dx = 0.f, Dy = 0.f, Dz = 0.f;   // per-lane div/curl sums
                if (a.nbr || DIVCURL || HASH) {
                    const float hinv = 1.f / h;
                    const float eL = eT + 2.f * rel * h;
                    const float hi2 = (h + eL) * (h + eL) * (1.f + 4.f * rel);
                    const float lo2 = h > eL ? (h - eL) * (h - eL) * (1.f - 4.f * rel) : 0.f;
                    double HH = -1.0;
                    const float4 vi = DIVCURL && okm ? a.vpack[pm] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const int kend = okm ? cm : 0;
                    int pos = 0;
                    for (int k = sub; __any_sync(0xffffffffu, k < kend); k += 4) {
                        bool in = false, xt = false;
                        int q = 0;
                        if (k < kend) {
                            const float x2 = mp.d[mm][k].x;
                            if (PART) q = jm[k];
                            if (x2 < hi2) {
                                q = jm[k];
                                in = x2 < lo2;
                                if (!in) {
                                    if (HH < 0.0) HH = wpp_hh(h, B);
                                    in = exact_pred(exact_d2(Xm, a.posm[q]), HH);
                                }
                            }
                            // an inactive near entry outside h_i with r_ij < h_j: an extra partner
                            if (PART && !in && a.flagp[q] == 0) xt = within_hj(a.list_xh[q]);
                        }
                        if (PART) add_extra(xt, q);
                        const unsigned nib = (__ballot_sync(0xffffffffu, in) >> (4 * mm)) & 0xfu;
                        if (in) {
                            const int kk = pos + __popc(nib & ((1u << sub) - 1u));
                            if (rec && kk < nnm) a.nbr[loff + kk] = q;
                            if (HASH) hs += splitmix64((unsigned long long)a.perm[q]);
                            if (DIVCURL) {
                                // d = x_j - x_i; r_ij = -d, v_ij = v_i - v_j
                                const uint4 Xj = a.posm[q];
                                const float dx = (float)(int)(Xj.x - Xm.x) * sf, dy = (float)(int)(Xj.y - Xm.y) * sf,
                                            dz = (float)(int)(Xj.z - Xm.z) * sf;
                                const float r2 = dx * dx + dy * dy + dz * dz;
                                if (r2 > 0.f) {   // coincident: no direction
                                    const float rinv = rsqrtf(r2);
                                    float w_, dw;
                                    spline<float>(r2 * rinv * hinv, w_, dw);
                                    const float4 vj = __ldg(a.vpack + q);
                                    const float gsc = vj.w * dw * rinv;
                                    const float vx = vi.x - vj.x, vy = vi.y - vj.y, vz = vi.z - vj.z;
                                    Dd -= gsc * (vx * dx + vy * dy + vz * dz);
                                    Dx -= gsc * (vy * dz - vz * dy);
                                    Dy -= gsc * (vz * dx - vx * dz);
                                    Dz -= gsc * (vx * dy - vy * dx);
                                }
                            }
                        }
                        pos += __popc(nib);
                    }
                    if (rec && pos != nnm) loff = -1;   // cannot happen: the same predicate counted nnm
                    if (PART) {
                        // the far entries: r_ij > h_i surely, partners when r_ij < h_j
                        const int kf = okm ? min(cf, kMpFar) : 0;
                        const int32_t* xm = mpx + mm * kMpFar;
                        for (int k = sub; __any_sync(0xffffffffu, k < kf); k += 4) {
                            bool xt = false;
                            int q = 0;
                            if (k < kf) {
                                q = xm[k];
                                xt = within_hj(a.list_xh[q]);
                            }
                            add_extra(xt, q);
                        }
                    }
                    if (HASH) {
                        hs += __shfl_xor_sync(0xffffffffu, hs, 1);
                        hs += __shfl_xor_sync(0xffffffffu, hs, 2);
                    }
                }
                if (DIVCURL) {
                    float cd, cx, cy, cz;
                    wpp_fold_quad2(Dd, cd, Dx, cx);
                    wpp_fold_quad2(Dy, cy, Dz, cz);
                    Dd = __fsub_rn(Dd, cd);
                    Dx = __fsub_rn(Dx, cx);
                    Dy = __fsub_rn(Dy, cy);
                    Dz = __fsub_rn(Dz, cz);
                }
                if (okm && sub == 0) {
                    const float smw = __fsub_rn(fSmw, Cmw), smdw = __fsub_rn(fSmdw, Cmdw);
                    const float rho = 2.5464790894703255f * smw * hinv_cube(h);   // 8/(pi h^3) sum m w
                    a.h[oim] = h;
                    a.rho[oim] = rho;
                    a.omega[oim] = smdw != 0.f ? -3.f * smw / smdw : 1.f;
                    a.n_ngb[oim] = nnm;
                    a.flags[oim] = (uint8_t)st;
                    if (HASH) a.hash[oim] = hs;
                    if (a.nbr) {
                        a.nbr_off[pm] = loff >= 0 ? (int)loff : 0;
                        a.nbr_n[pm] = loff >= 0 ? nnm : -1;
                        a.list_xh[pm] = make_uint4(Xm.x, Xm.y, Xm.z, __float_as_uint(h));
                        a.list_ep[pm] = gen;
                        if (PART) a.ext_n[pm] = cf > kMpFar || nex > kExtCap ? (unsigned)kExtCap + 1u : (unsigned)nex;
                        ++c_lists;
                    }
                    if (DIVCURL) {
                        // div = -(1/rho) sum m v_ij . grad W, curl = |(1/rho) sum m v_ij x grad W|,
                        // grad_i W = 8/(pi h^4) w'(q) r_ij / r
                        const float nr = 2.5464790894703255f * hinv_cube(h) / h / rho;
                        a.divv[oim] = -nr * Dd;
                        a.curlv[oim] = nr * sqrtf(Dx * Dx + Dy * Dy + Dz * Dz);
                    }
                    c_pairs += (unsigned)nnm;
                    c_status |= st;
                }
                // members for the one-particle path, from the h they reached
                const unsigned rb = __ballot_sync(0xffffffffu, rew && sub == 0);
                todo = 0;
#pragma unroll
                for (int k = 0; k < kMpMembers; ++k) todo |= ((rb >> (4 * k)) & 1u) << k;
                const float hnow = __shfl_sync(0xffffffffu, h, (int)(lane & 7u) * 4);
                if ((int)lane < G.n && ((todo >> lane) & 1u)) hl = hnow;
                __syncwarp();
            }
            // the members left over go to the one-particle kernel, each with the h
            // it should start from
            if (todo) {
                const int nl = __popc(todo);
                unsigned o = 0;
                if (lane == 0) o = atomicAdd(a.left_n, (unsigned)nl);
                o = __shfl_sync(0xffffffffu, o, 0);
                if ((int)lane < G.n && ((todo >> lane) & 1u)) {
                    a.left[o + __popc(todo & lt)] = G.p;
                    a.h[ol] = hl;
                    // PART: the one-particle kernel finds no far partners; the force pass walks for it
                    if (PART) a.ext_n[G.p] = (unsigned)kExtCap + 1u;
                }
            }
        }
    }
    // per-lane counters: lanes 4m hold the members', lane 0 the candidate tests
    c_pairs = warp_sum(c_pairs);
    c_evals = warp_sum(c_evals);
    c_lists = warp_sum(c_lists);
    c_tests = warp_sum(c_tests);
    c_status = __reduce_or_sync(0xffffffffu, c_status);
    if (lane == 0) {
        if (a.nbr && c_lists) atomicAdd(&a.list_st[0], c_lists);
        atomicAdd(&a.ctr->density_pairs, (unsigned long long)c_pairs);
        atomicAdd(&a.ctr->density_evals, (unsigned long long)c_evals);
        atomicAdd(&a.ctr->pair_tests, c_tests);
        if (c_status) atomicOr(&a.ctr->status, c_status);
    }
}

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
            const WppGroup G = wpp_group(a.boxes, a.n_boxes, a.act, t, t1, a.grp_shift);
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
                const float Rg = warp_max(a.fixed_h ? hl : hl * a.walk_r);
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
                        if (HH < 0.0) HH = wpp_hh(h, B);
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
                        Rw = a.fixed_h ? h : h * a.walk_r;
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
                            if (HHf < 0.0) HHf = wpp_hh(h, B);
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
                            a.list_xh[p] = make_uint4(Xi.x, Xi.y, Xi.z, __float_as_uint(h));
                            a.list_ep[p] = a.list_st[kListGen];
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
// h_i^2 and in FP64 inside it. The pair goes straight into i's fixed segment
// of kExtCap entries at the slot its counter hands out (scatter order); a
// count beyond kExtCap leaves the segment incomplete, which the sort marks.
// The pass is bound by the latency of its dependent loads (list head, list
// entries, then each entry's (X_i, h_i)), so a warp keeps three particles in
// flight: the head of the one after next, the first 64 entries of the next,
// and the gathers of the current one.
__global__ void __launch_bounds__(256) k_list_ext(const BoxDesc* __restrict__ boxes, int nb, int n,
                                                  const uint4* __restrict__ posm, const int32_t* __restrict__ nbr,
                                                  const int32_t* __restrict__ nbr_off,
                                                  const int32_t* __restrict__ nbr_n, const uint4* __restrict__ list_xh,
                                                  uint32_t* __restrict__ ext_n, int32_t* __restrict__ ext,
                                                  unsigned* list_st, const int32_t* __restrict__ act,
                                                  const uint32_t* __restrict__ count, const uint8_t* __restrict__ flag,
                                                  const uint32_t* __restrict__ list_ep) {
    // Every particle of the call must have had its list written, else the
    // extra lists cannot be completed: the active list (act given), or else
    // all n particles (the device count must then be n as well).
    const int na = (int)*count;
    const int nj = act ? na : n;
    if (list_st[0] != (unsigned)nj || (!act && na != n)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&list_st[1], 2u);
        return;
    }
    const unsigned gen = list_st[kListGen];
    const unsigned lane = lane_id();
    const int warps = gridDim.x * (blockDim.x >> 5);
    const float band = 9.5367431640625e-07f;  // 2^-20
    // a list head: the particle (-1 past the end), its list (count -2: not
    // recorded by this call, -1: missing) and its (X_j, h_j)
    struct Head {
        int j, cnt, off;
        uint4 X;
    };
    auto head = [&](int t) {
        Head hd = {-1, 0, 0, make_uint4(0u, 0u, 0u, 0u)};
        if (t < nj) {
            hd.j = act ? act[t] : t;
            hd.cnt = nbr_n[hd.j];
            hd.off = nbr_off[hd.j];
            hd.X = list_xh[hd.j];
            if (act && list_ep[hd.j] != gen) hd.cnt = -2;
        }
        return hd;
    };
    // its first 64 entries, two per lane
    auto first = [&](const Head& hd, int& i0, int& i1) {
        i0 = hd.j >= 0 && (int)lane < hd.cnt ? nbr[hd.off + (int)lane] : -1;
        i1 = hd.j >= 0 && (int)lane + 32 < hd.cnt ? nbr[hd.off + (int)lane + 32] : -1;
    };
    int t = blockIdx.x * (blockDim.x >> 5) + (int)(threadIdx.x >> 5);
    Head cur = head(t), nxt = head(t + warps);
    int i0, i1;
    first(cur, i0, i1);
    while (cur.j >= 0) {
        const Head far = head(t + 2 * warps);
        int n0, n1;
        first(nxt, n0, n1);
        const uint4 X0 = i0 >= 0 ? list_xh[i0] : make_uint4(0u, 0u, 0u, 0u);
        const uint4 X1 = i1 >= 0 ? list_xh[i1] : make_uint4(0u, 0u, 0u, 0u);
        if (cur.cnt < 0) {   // j's list is missing: the extra lists cannot be completed
            if (lane == 0) atomicOr(&list_st[1], 1u);
        } else {
            const int j = cur.j;
            const BoxDesc& B = boxes[nb == 1 ? 0 : wpp_box(boxes, nb, j)];
            const float Hs = B.Hs;   // integer units per box unit
            const uint4 Xj = cur.X;
            const float hj = __uint_as_float(Xj.w);
            auto decide = [&](uint4 Xi) {
                const float hi = __uint_as_float(Xi.w);
                bool x = false;
                if (hi < hj) {
                    const unsigned long long D2 = exact_d2(Xi, Xj);
                    const float d2 = __ull2float_rn(D2), Hi = hi * Hs, H2 = Hi * Hi;
                    if (d2 > H2 * (1.f + band)) x = true;
                    else if (!(d2 < H2 * (1.f - band))) x = !exact_pred(D2, wpp_hh(hi, B));
                }
                return x;
            };
            auto place = [&](int i) {
                if (act && !flag[i]) return;   // an inactive i: its extra partners are not needed
                const unsigned slot = atomicAdd(&ext_n[i], 1u);
                if (slot < (unsigned)kExtCap) ext[(size_t)i * kExtCap + slot] = j;
            };
            if (i0 >= 0 && decide(X0)) place(i0);
            if (i1 >= 0 && decide(X1)) place(i1);
            // entries past the first 64 (rare)
            for (int k = 64 + (int)lane; k < cur.cnt; k += 32) {
                const int i = nbr[cur.off + k];
                if (decide(list_xh[i])) place(i);
            }
        }
        t += warps;
        cur = nxt;
        nxt = far;
        i0 = n0;
        i1 = n1;
    }
}

// Extra-partner segments in ascending order, in place (the order fixes the
// force pass's sums): up to 64 entries each goes to its rank (registers), up
// to kExtCap through a bitonic sort in shared memory. A segment that
// overflowed is marked kExtUnusable, and the force pass walks for that
// particle. A warp reads the counts of 32 particles at a time and sorts their
// segments one after another.
__global__ void __launch_bounds__(256) k_list_sort(int n, int32_t* __restrict__ ext, uint32_t* __restrict__ ext_n,
                                                   const unsigned* __restrict__ list_st,
                                                   const int32_t* __restrict__ act, const uint32_t* __restrict__ count) {
    if (list_st[1] != 0u) return;   // the lists cannot serve a force call
    __shared__ int buf[8][kExtCap];
    int* sb = buf[threadIdx.x >> 5];
    const unsigned lane = lane_id();
    const int warps = gridDim.x * (blockDim.x >> 5);
    const int ni = act ? (int)*count : n;
    for (int t0 = (blockIdx.x * (blockDim.x >> 5) + (int)(threadIdx.x >> 5)) * 32; t0 < ni; t0 += warps * 32) {
        const int tl = t0 + (int)lane;
        const int il = tl < ni ? (act ? act[tl] : tl) : -1;
        const unsigned cl = il >= 0 ? ext_n[il] : 0u;
        if (cl > (unsigned)kExtCap) ext_n[il] = kExtUnusable;
        unsigned todo = __ballot_sync(0xffffffffu, cl >= 2u && cl <= (unsigned)kExtCap);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1u;
            const int i = __shfl_sync(0xffffffffu, il, src);
            const int c = (int)__shfl_sync(0xffffffffu, cl, src);
            int32_t* seg = ext + (size_t)i * kExtCap;
            if (c <= 32) {   // one entry per lane: its rank among the c
                const int v0 = (int)lane < c ? seg[lane] : 0x7fffffff;
                int r0 = 0;
                for (int k = 0; k < c; ++k) r0 += __shfl_sync(0xffffffffu, v0, k) < v0;
                __syncwarp();   // every lane has read the segment before it is overwritten
                if ((int)lane < c) seg[r0] = v0;
            } else if (c <= 64) {
                const int v0 = (int)lane < c ? seg[lane] : 0x7fffffff;
                const int v1 = (int)lane + 32 < c ? seg[lane + 32] : 0x7fffffff;
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
                __syncwarp();   // every lane has read the segment before it is overwritten
                if ((int)lane < c) seg[r0] = v0;
                if ((int)lane + 32 < c) seg[r1] = v1;
            } else {
                constexpr int P = kExtCap;   // a power of two
                for (int k = (int)lane; k < P; k += 32) sb[k] = k < c ? seg[k] : 0x7fffffff;
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
                for (int k = (int)lane; k < c; k += 32) seg[k] = sb[k];
            }
            __syncwarp();
        }
    }
}

// Start of a density call that records lists: clear the status words, one
// more generation (the stamp of the lists this call writes).
__global__ void k_list_begin(unsigned* list_st) {
    const int t = (int)threadIdx.x;
    if (t < kListGen) list_st[t] = 0u;
    else if (t == kListGen) list_st[kListGen] += 1u;
}

// A call on part of the particles: the h every inactive particle keeps (with
// its position, in sorted order) for the extra-partner tests, and the h of
// the inactive particles alone in caller order (0 for the active ones) for the
// node h_max that bounds where such partners can be.
__global__ void k_list_snap(int n, const int32_t* __restrict__ perm, const float* __restrict__ h,
                            const uint4* __restrict__ posm, const uint8_t* __restrict__ flag,
                            uint4* __restrict__ list_xh, float* __restrict__ h_inactive) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int o = perm[p];
    const float hp = h[o];
    const uint4 X = posm[p];
    list_xh[p] = make_uint4(X.x, X.y, X.z, __float_as_uint(hp));
    h_inactive[o] = flag[p] ? 0.f : hp;
}

// Sorted (v, m) for the density pass's velocity divergence and curl.
__global__ void k_vel_pack(int n, const int32_t* __restrict__ perm, const float* __restrict__ vel,
                           const float4* __restrict__ posf, float4* __restrict__ vm) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const size_t o = (size_t)perm[p];
    vm[p] = make_float4(vel[3 * o], vel[3 * o + 1], vel[3 * o + 2], posf[p].w);
}

cudaError_t launch_density_wpp(sph_ctx* ctx, const DensityLaunch& a, int64_t n_active, cudaStream_t s) {
    sph_grid* g = const_cast<sph_grid*>(a.g);
    cudaError_t e = cudaMemsetAsync(ctx->queue + 2, 0, sizeof(unsigned), s);
    if (e) return e;
    WppArgs c = wpp_common(ctx, g, ctx->queue + 2);
    int blocks = 0;
    const int bps = std::min(a.blocks_per_sm > 0 ? a.blocks_per_sm : kWppDensityBps, kWppDensityMaxBps);
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
    c.walk_r = a.walk_radius > 0.0 ? (float)a.walk_radius : kWppWalkR;
    c.grp_shift = wpp_grp_shift(a.group_span);
    // the scratch holds kMpWarpsPerSm warps per SM of the device the grid was built on
    c.mp_j = g->ctx->sm_count >= ctx->sm_count ? g->mp_j : nullptr;
    if (a.divv) {
        k_vel_pack<<<(int)((g->n + 255) / 256), 256, 0, s>>>((int)g->n, g->perm, a.vel, g->posf, g->fvm);
        ++ctx->launches;
        c.vpack = g->fvm;
        c.divv = a.divv;
        c.curlv = a.curlv;
    }
    // Neighbour lists for the force pass, each stamped with this call's
    // generation. A call whose active set can cover every particle (no list,
    // or a list of n entries) records them whatever the kernel; they serve a
    // force call only if every particle was in fact active (checked on the
    // device: the list count and the lists written both equal n). With
    // SPH_PARTIAL_LISTS, a call on an active list (padded or not) that runs the
    // member-parallel kernel records the active particles' lists and also
    // finds their extra partners among the inactive ones.
    // (The partial lists need the member-parallel kernel: with the flag it runs
    // for any active set that is not too sparse to form groups.)
    const bool want_part = g->nbr != nullptr && a.active_list && a.partial_lists && n_active * 256 >= g->n;
    const bool mp_path = (want_part || wpp_groups_pay(ctx, n_active, g->n)) && c.mp_j != nullptr;
    const bool part = want_part && mp_path;
    const bool rec = part || (g->nbr != nullptr && n_active == g->n);
    if (rec) {
        c.nbr = g->nbr;
        c.nbr_off = g->nbr_off;
        c.nbr_n = g->nbr_n;
        c.list_xh = g->list_xh;
        c.list_st = g->list_st;
        c.list_ep = g->list_ep;
        c.ext = g->ext;
        c.ext_n = g->ext_n;
        c.list_pool = g->list_pool;
        // chunks small enough that every warp's first reservations fit in a quarter of the pool
        const long long warps = (long long)blocks * kWppWarps;
        c.list_chunk = (int)std::max<long long>(32, std::min<long long>(kListChunk, g->list_pool / (4 * warps)));
        k_list_begin<<<1, 32, 0, s>>>(g->list_st);
        ++ctx->launches;
        if ((e = cudaMemsetAsync(g->ext_n, 0, sizeof(uint32_t) * g->n, s))) return e;
        if (part) {
            const int n = (int)g->n;
            k_list_snap<<<(n + 255) / 256, 256, 0, s>>>(n, g->perm, a.h, g->posm, g->flag, g->list_xh, g->st_lo);
            ++ctx->launches;
            grid_refresh_hmax(g, g->st_lo, s);
            c.flagp = g->flag;
            c.mp_x = g->mp_x;
        }
    }
    WppSpan sp;
    if ((e = span_begin(ctx, a.time_kernels, 0, s, sp))) return e;
    const bool dc = a.divv != nullptr;
    if (!mp_path) {
        // sparse active sets form groups of one: the one-particle kernel alone
        auto k1 = a.hash ? (dc ? k_density_wpp<true, kWppLeftBps, true> : k_density_wpp<true, kWppLeftBps, false>)
                         : (dc ? k_density_wpp<false, kWppLeftBps, true> : k_density_wpp<false, kWppLeftBps, false>);
        int b1 = 0;
        wpp_shape(ctx, kWppLeftBps, n_active, b1, c.chunk);
        k1<<<b1, kWppThreads, 0, s>>>(c);
        ++ctx->launches;
    } else {
        // leftovers of the member-parallel kernel: list g->den_left, count queue[6],
        // work queue queue[5]
        if ((e = cudaMemsetAsync(ctx->queue + 5, 0, 2 * sizeof(unsigned), s))) return e;
        c.left = g->den_left;
        c.left_n = ctx->queue + 6;
        // whole groups per queue grab, whatever the active count: a warp's
        // group costs little more than one particle (the leftover kernel below
        // takes one particle at a time)
        c.chunk = kMpMembers;
        // 4 or 5 resident blocks (the shared memory of a block holds the member
        // near lists: 5 blocks fill an SM), 128 or 96 registers
        auto kd = part ? (bps <= 4 ? (a.hash ? (dc ? k_density_mp<true, 4, true, true> : k_density_mp<true, 4, false, true>)
                                            : (dc ? k_density_mp<false, 4, true, true> : k_density_mp<false, 4, false, true>))
                                  : (a.hash ? (dc ? k_density_mp<true, 5, true, true> : k_density_mp<true, 5, false, true>)
                                            : (dc ? k_density_mp<false, 5, true, true> : k_density_mp<false, 5, false, true>)))
                       : (bps <= 4 ? (a.hash ? (dc ? k_density_mp<true, 4, true, false> : k_density_mp<true, 4, false, false>)
                                            : (dc ? k_density_mp<false, 4, true, false> : k_density_mp<false, 4, false, false>))
                                  : (a.hash ? (dc ? k_density_mp<true, 5, true, false> : k_density_mp<true, 5, false, false>)
                                            : (dc ? k_density_mp<false, 5, true, false> : k_density_mp<false, 5, false, false>)));
        kd<<<blocks, kWppThreads, 0, s>>>(c);
        // the leftovers, one particle per warp (count on the device), from the h the
        // member-parallel kernel left for them
        WppArgs cl = c;
        cl.act = g->den_left;
        cl.count_ptr = ctx->queue + 6;
        cl.queue = ctx->queue + 5;
        cl.chunk = 1;
        cl.guess_h = 0;
        // each list reserved alone: the leftovers are few and scattered over
        // the warps, and a pool chunk per warp would be mostly unused
        cl.list_chunk = 0;
        int lblocks = 0, lchunk = 0;
        wpp_shape(ctx, kWppLeftBps, n_active, lblocks, lchunk);
        auto kl = a.hash ? (dc ? k_density_wpp<true, kWppLeftBps, true> : k_density_wpp<true, kWppLeftBps, false>)
                         : (dc ? k_density_wpp<false, kWppLeftBps, true> : k_density_wpp<false, kWppLeftBps, false>);
        kl<<<lblocks, kWppThreads, 0, s>>>(cl);
        ctx->launches += 2;
    }
    // SPH_TIME_KERNELS times the density kernel alone; the list build follows
    if ((e = span_end(ctx, sp, s))) return e;
    if (rec) {
        const int n = (int)g->n, hb = helper_blocks(ctx, n);
        const int32_t* act = part ? g->act : nullptr;
        const uint32_t* count = g->scan + n;
        k_list_ext<<<hb, 256, 0, s>>>(g->boxes, g->n_boxes, n, g->posm, g->nbr, g->nbr_off, g->nbr_n, g->list_xh,
                                      g->ext_n, g->ext, g->list_st, act, count, g->flag, g->list_ep);
        k_list_sort<<<hb, 256, 0, s>>>(n, g->ext, g->ext_n, g->list_st, act, count);
        ctx->launches += 2;
    }
    g->lists_rec = rec;
    return cudaGetLastError();
}

}  // namespace sph
