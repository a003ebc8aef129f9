// wpp_density.cu -- the default density pass (k_density_wpp) and the neighbour-list
// build that lets the force pass reuse its pair sets (k_list_ext, k_list_sort).
#include "wpp.cuh"

namespace sph {

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
__global__ void __launch_bounds__(256) k_list_ext(const BoxDesc* __restrict__ boxes, int nb, int n,
                                                  const uint4* __restrict__ posm, const int32_t* __restrict__ nbr,
                                                  const int32_t* __restrict__ nbr_off,
                                                  const int32_t* __restrict__ nbr_n, const float* __restrict__ list_h,
                                                  uint32_t* __restrict__ ext_n, int32_t* __restrict__ ext,
                                                  unsigned* list_st) {
    const unsigned lane = lane_id();
    const int warps = gridDim.x * (blockDim.x >> 5);
    const float band = 9.5367431640625e-07f;  // 2^-20
    for (int j = blockIdx.x * (blockDim.x >> 5) + (int)(threadIdx.x >> 5); j < n; j += warps) {
        const int cnt = nbr_n[j];
        if (cnt < 0) {   // j's list is missing: the extra lists cannot be completed
            if (lane == 0) atomicOr(&list_st[1], 1u);
            continue;
        }
        const int32_t* lj = nbr + nbr_off[j];
        const BoxDesc& B = boxes[nb == 1 ? 0 : wpp_box(boxes, nb, j)];
        const float Hs = B.Hs;   // integer units per box unit
        const uint4 Xj = posm[j];
        const float hj = list_h[j];
        auto decide = [&](float hi, uint4 Xi) {
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
            const unsigned slot = atomicAdd(&ext_n[i], 1u);
            if (slot < (unsigned)kExtCap) ext[(size_t)i * kExtCap + slot] = j;
        };
        // two entries per lane per step (k and k + 32), their gathers issued together
        for (int k = (int)lane; k < cnt; k += 64) {
            const int k1 = k + 32;
            const bool two = k1 < cnt;
            const int i0 = lj[k], i1 = two ? lj[k1] : i0;
            const float h0 = list_h[i0], h1 = list_h[i1];
            const uint4 X0 = h0 < hj ? posm[i0] : Xj, X1 = (two && h1 < hj) ? posm[i1] : Xj;
            if (decide(h0, X0)) place(i0);
            if (two && decide(h1, X1)) place(i1);
        }
    }
}

// Warp per particle: its extra partners (distinct indices) in ascending order,
// in place in its segment: up to 64 entries each goes to its rank (registers),
// up to kExtCap through a bitonic sort in shared memory. A segment that
// overflowed is marked kExtUnusable, and the force pass walks for that particle.
__global__ void __launch_bounds__(256) k_list_sort(int n, int32_t* __restrict__ ext, uint32_t* __restrict__ ext_n) {
    __shared__ int buf[8][kExtCap];
    int* sb = buf[threadIdx.x >> 5];
    const unsigned lane = lane_id();
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (int)(threadIdx.x >> 5); i < n; i += warps) {
        const unsigned cu = ext_n[i];
        if (cu > (unsigned)kExtCap) {
            if (lane == 0) ext_n[i] = kExtUnusable;
            continue;
        }
        const int c = (int)cu;
        if (c < 2) continue;
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
              : bps == 7 ? (a.hash ? (dc ? k_density_wpp<true, 7, true> : k_density_wpp<true, 7, false>)
                                   : (dc ? k_density_wpp<false, 7, true> : k_density_wpp<false, 7, false>))
                         : (a.hash ? (dc ? k_density_wpp<true, 8, true> : k_density_wpp<true, 8, false>)
                                   : (dc ? k_density_wpp<false, 8, true> : k_density_wpp<false, 8, false>));
    kd<<<blocks, kWppThreads, 0, s>>>(c);
    ++ctx->launches;
    // SPH_TIME_KERNELS times the density kernel alone; the list build follows
    if ((e = span_end(ctx, sp, s))) return e;
    if (full) {
        const int n = (int)g->n, hb = helper_blocks(ctx, n);
        if ((e = cudaMemsetAsync(g->ext_n, 0, sizeof(uint32_t) * n, s))) return e;
        k_list_ext<<<hb, 256, 0, s>>>(g->boxes, g->n_boxes, n, g->posm, g->nbr, g->nbr_off, g->nbr_n, g->list_h,
                                      g->ext_n, g->ext, g->list_st);
        k_list_sort<<<hb, 256, 0, s>>>(n, g->ext, g->ext_n);
        ctx->launches += 2;
    }
    g->lists_full = full;
    return cudaGetLastError();
}

}  // namespace sph
