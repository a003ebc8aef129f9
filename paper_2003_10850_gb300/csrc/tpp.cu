// tpp.cu -- thread-per-particle density and force kernels (SPH_PER_THREAD_WALK,
// and SPH_FP64 for the plain method in double; the default path is the
// warp-per-group kernels of wpp_density.cu and wpp_force.cu), and the force
// pass's per-particle packing (k_force_pack) that every force path reads.
//
// One thread per active particle, consecutive threads on Morton-consecutive
// particles, each walking the hierarchy depth-first with its own radius, so a
// particle only tests candidates whose leaf box its own sphere reaches (the
// paper's per-particle tree walk, Sec. 1, done on the GPU). Versus the plain
// FP32 baseline (plain.cu):
//   * the h iteration runs inside the kernel (FP64 Newton on N^(1/3) with a
//     bracket, per thread), no host round trip per iteration;
//   * candidate positions come as FP32 offsets from their leaf's centre,
//     precomputed at grid build, so a pair costs three adds instead of three
//     integer-to-float conversions;
//   * sums are compensated (Kahan) per leaf, du/dt accumulated in FP64;
//   * the neighbour predicate is exact ((double)D2 < H^2 on integer
//     coordinates) inside a thin band around the FP32 radius test;
//   * force candidates are read from packed per-call float4 records.
// T = double runs the same walk with FP64 pair arithmetic on exact integer
// separations.
#include <type_traits>

#include "internal.cuh"

namespace sph {

constexpr int kTppThreads = 128;
constexpr int kTppStack = 96;   // depth-first: <= 7 pending siblings per level + 1

template <typename T>
struct TBand;
template <>
struct TBand<float> {
    static constexpr float rel = 9.5367431640625e-07f;  // 2^-20
};
template <>
struct TBand<double> {
    static constexpr double rel = 1.7763568394002505e-15;  // 2^-49
};

__device__ __forceinline__ int tpp_box_of(const BoxDesc* boxes, int nb, long long p) {
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (boxes[mid].off <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Child test: periodic distance from the particle to the node box below R.
// The FP32 offset of the node centre is rounded by at most 2^-23 of its size,
// which the slack covers.
__device__ __forceinline__ bool tpp_node_near(uint4 c, float4 e, uint4 X, float sf, float R) {
    const float dx = (float)(int)(c.x - X.x) * sf, dy = (float)(int)(c.y - X.y) * sf,
                dz = (float)(int)(c.z - X.z) * sf;
    const float gx = fmaxf(fabsf(dx) - e.x, 0.f), gy = fmaxf(fabsf(dy) - e.y, 0.f),
                gz = fmaxf(fabsf(dz) - e.z, 0.f);
    const float Rt = R * (1.f + 3.0517578125e-05f) +
                     2.384185791015625e-07f * (fabsf(dx) + fabsf(dy) + fabsf(dz)) + 4.f * sf;
    return gx * gx + gy * gy + gz * gz < Rt * Rt;
}

template <typename T>
__device__ __forceinline__ T tpp_sqrt(T x) {
    if constexpr (std::is_same<T, float>::value) return x > 0.f ? x * rsqrtf(x) : 0.f;
    else return sqrt(x);
}


// One bracketed step of the smoothing-length solve. f = N - N_t arrives in
// FP64 (from the compensated FP32 sums); the bracket and the new h are kept in
// FP64, while the Newton step on N^(1/3) - N_t^(1/3) is formed in FP32 (it is
// a correction, and FP64 cbrt/division would cost ~60 FP32 slots each on this
// part). Returns false when h cannot move (converged to the float grid or an
// error bit was set).
__device__ __forceinline__ bool h_update(float& h, double f, float N, float dN, float n_target, double cap,
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
        // outside the bracket, or not converging fast (the step did not halve):
        // bisect (the safeguard of Newton-Raphson with bracketing)
        hn = 0.5 * (blo + bhi);
    }
    dold = fabsf((float)(hn - (double)h));
    float hf = (float)hn;
    if (!(hf > (float)blo) || (!isinf(bhi) && !(hf < (float)bhi))) {
        const float mid = (float)(0.5 * (blo + bhi));
        hf = (mid > (float)blo && mid < (float)bhi) ? mid : h;
    }
    if (hf == h) return false;  // the bracket is one float wide: h is the best float
    h = hf;
    return true;
}

// ---------------------------------------------------------------------------
// Density
// ---------------------------------------------------------------------------

struct TppDensArgs {
    const BoxDesc* boxes;
    int n_boxes;
    const int32_t* act;
    const int* count_ptr;   // device count (subset), or NULL
    int count;
    const uint4* posm;
    const float4* posf;
    const int32_t* perm;
    const uint4* node_c;
    const float4* node_e;
    const uint4* node_lo;
    const uint4* node_hi;
    float* h;
    float* rho;
    float* omega;
    int32_t* n_ngb;
    uint8_t* flags;
    unsigned long long* hash;
    double n_target, n_tol;
    int max_iter;
    int fixed_h, guess_h;
    Counters* ctr;
};

template <typename T>
struct TppDSums {
    T sw, cw, sdw, cdw, smw, cmw, smdw, cmdw;
    int nn;
    unsigned long long hs, tests;
};

template <typename T, bool HASH>
__device__ __forceinline__ void tpp_density_walk(const TppDensArgs& a, const BoxDesc& B, int p, uint4 Xi,
                                                 float h, TppDSums<T>& S) {
    double HH = -1.0;  // (h 2^32/L)^2, formed on the first band pair only
    const double s = ldexp(B.L, -32);
    const float sf = (float)s;
    const T sT = (T)s;
    const T hT = (T)h, hinv = T(1) / hT;
    int stack[kTppStack];
    int sp = 0;
    stack[sp++] = B.nlev == 1 ? 0 : (B.nlev - 1) << 27;
    const long long pend = B.off + B.n;
    while (sp > 0) {
        const int enc = stack[--sp];
        const int lev = enc >> 27, t = enc & ((1 << 27) - 1);
        if (lev > 0) {
            const int cl = lev - 1;
            const int c0 = t * kFan, c1 = min(c0 + kFan, B.lvl_n[cl]);
            const int base = B.lvl_off[cl];
            for (int c = c0; c < c1; ++c)
                if (tpp_node_near(a.node_c[base + c], a.node_e[base + c], Xi, sf, h)) stack[sp++] = (cl << 27) | c;
            continue;
        }
        // leaf t: its particles' offsets from the leaf centre are in posf
        const int nd = B.lvl_off[0] + t;
        const uint4 C = a.node_c[nd];
        const float4 E = a.node_e[nd];
        const T ox = (T)(int)(C.x - Xi.x) * sT, oy = (T)(int)(C.y - Xi.y) * sT, oz = (T)(int)(C.z - Xi.z) * sT;
        // rounding bound of r for pairs in this leaf, and the predicate band
        const T eL = TBand<T>::rel * (T(4) * (T)(E.x + E.y + E.z) + T(2) * (fabs(ox) + fabs(oy) + fabs(oz)) + T(2) * hT);
        const T lo2 = hT > eL ? (hT - eL) * (hT - eL) * (T(1) - T(4) * TBand<T>::rel) : T(0);
        const T hi2 = (hT + eL) * (hT + eL) * (T(1) + T(4) * TBand<T>::rel);
        const long long q0 = B.off + (long long)t * kLeaf, q1 = min(q0 + kLeaf, pend);
        // A leaf straddling a large Morton jump can be wider than half the box;
        // then centre offset + in-leaf offset is not the minimum image and the
        // pair uses the exact integer separation instead.
        const bool wide = T(2) * (T)(E.x + E.y + E.z) + hT >= T(0.45) * (T)B.L;
        T pw = 0, pdw = 0, pmw = 0, pmdw = 0;
        for (long long q = q0; q < q1; ++q) {
            T dx, dy, dz, m;
            if (std::is_same<T, float>::value && !wide) {
                const float4 f = a.posf[q];
                dx = ox + f.x; dy = oy + f.y; dz = oz + f.z; m = f.w;
            } else {
                const uint4 Xj = a.posm[q];
                dx = (T)(int)(Xj.x - Xi.x) * sT; dy = (T)(int)(Xj.y - Xi.y) * sT; dz = (T)(int)(Xj.z - Xi.z) * sT;
                m = (T)__uint_as_float(Xj.w);
            }
            const T r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < hi2) {
                bool in = r2 < lo2;
                if (!in) {
                    if (HH < 0.0) {
                        const double Hd = (double)h * 4294967296.0 / B.L;
                        HH = Hd * Hd;
                    }
                    in = exact_pred(exact_d2(Xi, a.posm[q]), HH);
                }
                if (in) {
                    const T qq = tpp_sqrt<T>(r2) * hinv;
                    T w, dw;
                    spline<T>(qq, w, dw);
                    const T qdw = qq * dw;
                    pw += w;
                    pdw += qdw;
                    pmw += m * w;
                    pmdw += m * qdw;
                    if (q != p) {
                        ++S.nn;
                        if (HASH) S.hs += splitmix64((unsigned long long)a.perm[q]);
                    }
                }
            }
        }
        S.tests += (unsigned long long)(q1 - q0);
        kahan_add(S.sw, S.cw, pw);
        kahan_add(S.sdw, S.cdw, pdw);
        kahan_add(S.smw, S.cmw, pmw);
        kahan_add(S.smdw, S.cmdw, pmdw);
    }
}

__device__ float tpp_guess_h(const BoxDesc& B, const uint4* node_lo, const uint4* node_hi, long long p, double s,
                             double n_target) {
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

template <typename T, bool HASH>
__global__ void __launch_bounds__(kTppThreads) k_density_tpp(TppDensArgs a) {
    const int cnt = a.count_ptr ? *a.count_ptr : a.count;
    unsigned long long c_pairs = 0, c_evals = 0, c_tests = 0;
    unsigned c_status = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
        const int p = a.act[t];
        const BoxDesc& B = a.boxes[a.n_boxes == 1 ? 0 : tpp_box_of(a.boxes, a.n_boxes, p)];
        const double L = B.L, s = ldexp(L, -32);
        const uint4 Xi = a.posm[p];
        const int oi = a.perm[p];
        float h = a.h[oi];
        if (a.guess_h || !(h > 0.f) || !isfinite(h)) h = tpp_guess_h(B, a.node_lo, a.node_hi, p, s, a.n_target);
        const double cap = 0.5 * L * (1.0 - 1e-9);
        double blo = 0.0, bhi = INFINITY;
        float dold = INFINITY;
        unsigned st = 0;
        TppDSums<T> S;
        for (int it = 0;; ++it) {
            S.sw = S.cw = S.sdw = S.cdw = S.smw = S.cmw = S.smdw = S.cmdw = 0;
            S.nn = 0;
            S.hs = 0;
            S.tests = 0;
            tpp_density_walk<T, HASH>(a, B, p, Xi, h, S);
            ++c_evals;
            c_tests += S.tests;
            const double f = (32.0 / 3.0) * ((double)S.sw - (double)S.cw) - a.n_target;
            if (a.fixed_h || fabs(f) <= a.n_tol) break;
            if (it >= a.max_iter) { st |= ST_NOT_CONVERGED; break; }
            const float N = (float)((32.0 / 3.0) * ((double)S.sw - (double)S.cw));
            const float dN = -(32.f / 3.f) * (float)((double)S.sdw - (double)S.cdw) / h;
            if (!h_update(h, f, N, dN, (float)a.n_target, cap, blo, bhi, dold, st)) break;
        }
        const double smw = (double)S.smw - (double)S.cmw, smdw = (double)S.smdw - (double)S.cmdw;
        const double hd = (double)h;
        a.h[oi] = h;
        a.rho[oi] = (float)(8.0 / (3.141592653589793 * hd * hd * hd) * smw);
        a.omega[oi] = (float)(smdw != 0.0 ? -3.0 * smw / smdw : 1.0);
        a.n_ngb[oi] = S.nn;
        a.flags[oi] = (uint8_t)st;
        if (HASH) a.hash[oi] = S.hs;
        c_pairs += (unsigned long long)S.nn;
        c_status |= st;
    }
    c_pairs = warp_sum(c_pairs);
    c_evals = warp_sum(c_evals);
    c_tests = warp_sum(c_tests);
    c_status = __reduce_or_sync(0xffffffffu, c_status);
    if (lane_id() == 0) {
        atomicAdd(&a.ctr->density_pairs, c_pairs);
        atomicAdd(&a.ctr->density_evals, c_evals);
        atomicAdd(&a.ctr->pair_tests, c_tests);
        if (c_status) atomicOr(&a.ctr->status, c_status);
    }
}

// ---------------------------------------------------------------------------
// Buffered density (FP32 default): one walk per particle, iterations on a
// per-thread buffer of (r^2, m) for every candidate within the walk radius
// R = 1.06 h. N_eff is number-weighted, so each Newton step only re-sums
// w(sqrt(r^2)/h) over the buffer; the walk is repeated only when the root
// leaves [0, R). Particles whose buffer overflows, or whose final sums have a
// pair inside the FP32 predicate band, are finished by the exact per-walk
// loop (tpp_density_walk) at the h reached.
// ---------------------------------------------------------------------------

constexpr int kDensBuf = 96;
constexpr float kWalkMargin = 1.06f;

// Depth-first walk in "while-while" form: descend until this thread holds a
// leaf (or has nothing left), then process it. The leaf work, the costly
// part, runs with the warp reconverged instead of interleaved with node tests.
template <class LeafFn>
__device__ __forceinline__ void tpp_walk_leaves(const BoxDesc& B, const uint4* __restrict__ node_c,
                                                const float4* __restrict__ node_e, uint4 Xi, float sf, float R,
                                                bool use_hmax, LeafFn&& leaf) {
    int stack[kTppStack];
    int sp = 0;
    stack[sp++] = B.nlev == 1 ? 0 : (B.nlev - 1) << 27;
    for (;;) {
        int lt = -1;
        while (sp > 0) {
            const int enc = stack[--sp];
            const int lev = enc >> 27, t = enc & ((1 << 27) - 1);
            if (lev == 0) {
                lt = t;
                break;
            }
            const int cl = lev - 1;
            const int c0 = t * kFan, c1 = min(c0 + kFan, B.lvl_n[cl]);
            const int base = B.lvl_off[cl];
            for (int c = c0; c < c1; ++c) {
                const float4 e = node_e[base + c];
                if (tpp_node_near(node_c[base + c], e, Xi, sf, use_hmax ? fmaxf(R, e.w) : R))
                    stack[sp++] = (cl << 27) | c;
            }
        }
        if (lt < 0) break;
        leaf(lt);
    }
}

template <bool HASH>
__global__ void __launch_bounds__(kTppThreads) k_density_buf(TppDensArgs a) {
    const int cnt_all = a.count_ptr ? *a.count_ptr : a.count;
    unsigned long long c_pairs = 0, c_evals = 0, c_tests = 0;
    unsigned c_status = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt_all; t += gridDim.x * blockDim.x) {
        const int p = a.act[t];
        const BoxDesc& B = a.boxes[a.n_boxes == 1 ? 0 : tpp_box_of(a.boxes, a.n_boxes, p)];
        const double L = B.L, s = ldexp(L, -32);
        const float sf = (float)s;
        const uint4 Xi = a.posm[p];
        const int oi = a.perm[p];
        float h = a.h[oi];
        if (a.guess_h || !(h > 0.f) || !isfinite(h)) h = tpp_guess_h(B, a.node_lo, a.node_hi, p, s, a.n_target);
        const double cap = 0.5 * L * (1.0 - 1e-9);
        double blo = 0.0, bhi = INFINITY;
        float dold = INFINITY;
        unsigned st = 0;
        bool exact_finish = false, finished = false;
        float2 buf[kDensBuf];
        int it = 0;
        double smw = 0.0, smdw = 0.0;
        int nn = 0;
        while (!finished) {
            // walk once with radius R, buffering every candidate inside it
            const float R = fminf(h * kWalkMargin, (float)cap);
            int nb = 0;
            float emax = 0.f;  // largest FP32 error bound of r over the leaves that fed the buffer
            unsigned long long tests = 0;
            tpp_walk_leaves(B, a.node_c, a.node_e, Xi, sf, R, false, [&](int lt) {
                const int nd = B.lvl_off[0] + lt;
                const uint4 C = a.node_c[nd];
                const float4 E = a.node_e[nd];
                const long long q0 = B.off + (long long)lt * kLeaf, q1 = min(q0 + kLeaf, B.off + B.n);
                const bool wide = 2.f * (E.x + E.y + E.z) + R >= 0.45f * (float)B.L;
                const float ox = (float)(int)(C.x - Xi.x) * sf, oy = (float)(int)(C.y - Xi.y) * sf,
                            oz = (float)(int)(C.z - Xi.z) * sf;
                // bound on the FP32 error of r for pairs in this leaf (as in tpp_density_walk)
                const float eL = 9.5367431640625e-07f *
                                 (4.f * (E.x + E.y + E.z) + 2.f * (fabsf(ox) + fabsf(oy) + fabsf(oz)));
                const float Rb = R * (1.f + 3.814697265625e-06f) + eL;
                const float Rb2 = Rb * Rb;
                bool fed = false;
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
                    if (r2 < Rb2) {
                        if (nb < kDensBuf) buf[nb] = make_float2(r2, m);
                        ++nb;
                        fed = true;
                    }
                }
                if (fed) emax = fmaxf(emax, eL);
                tests += (unsigned long long)(q1 - q0);
            });
            c_tests += tests;
            if (nb > kDensBuf) {  // too many candidates to buffer
                exact_finish = true;
                break;
            }
            // Newton/bisection on the buffer until converged or the root leaves [0, R)
            for (;;) {
                const float hinv = 1.f / h, h2 = h * h;
                float Sw = 0.f, Cw = 0.f, Sdw = 0.f, Cdw = 0.f;
                for (int k0 = 0; k0 < nb; k0 += 8) {
                    float pw = 0.f, pdw = 0.f;
                    const int k1 = min(k0 + 8, nb);
                    for (int k = k0; k < k1; ++k) {
                        const float r2 = buf[k].x;
                        if (r2 < h2) {
                            const float qq = (r2 > 0.f ? r2 * rsqrtf(r2) : 0.f) * hinv;
                            float w, dw;
                            spline<float>(qq, w, dw);
                            pw += w;
                            pdw += qq * dw;
                        }
                    }
                    kahan_add(Sw, Cw, pw);
                    kahan_add(Sdw, Cdw, pdw);
                }
                ++c_evals;
                const double f = (32.0 / 3.0) * ((double)Sw - (double)Cw) - a.n_target;
                if (fabs(f) <= a.n_tol) { finished = true; break; }
                if (it >= a.max_iter) { st |= ST_NOT_CONVERGED; finished = true; break; }
                ++it;
                const float N = (32.f / 3.f) * (Sw - Cw);
                const float dN = -(32.f / 3.f) * (Sdw - Cdw) / h;
                if (!h_update(h, f, N, dN, (float)a.n_target, cap, blo, bhi, dold, st)) { finished = true; break; }
                if (h >= R * (1.f - 1.52587890625e-05f)) break;  // outside the buffer: walk again
            }
            if (!finished) continue;
            // final mass-weighted sums and neighbour count at h; a pair inside
            // the FP32 band of the exact predicate sends the particle to the
            // exact walk
            const float hinv = 1.f / h;
            const float eb = emax + 1.9073486328125e-06f * h;  // + 2^-19 h, as the exact walk's band
            const float lo2 = h > eb ? (h - eb) * (h - eb) * (1.f - 3.814697265625e-06f) : 0.f;
            const float hi2 = (h + eb) * (h + eb) * (1.f + 3.814697265625e-06f);
            float Smw = 0.f, Cmw = 0.f, Smdw = 0.f, Cmdw = 0.f;
            int n_in = 0;
            bool band = false;
            for (int k0 = 0; k0 < nb; k0 += 8) {
                float pmw = 0.f, pmdw = 0.f;
                const int k1 = min(k0 + 8, nb);
                for (int k = k0; k < k1; ++k) {
                    const float2 e = buf[k];
                    if (e.x < hi2) {
                        if (e.x >= lo2) band = true;
                        const float qq = (e.x > 0.f ? e.x * rsqrtf(e.x) : 0.f) * hinv;
                        float w, dw;
                        spline<float>(qq, w, dw);
                        pmw += e.y * w;
                        pmdw += e.y * qq * dw;
                        ++n_in;
                    }
                }
                kahan_add(Smw, Cmw, pmw);
                kahan_add(Smdw, Cmdw, pmdw);
            }
            if (band) { exact_finish = true; break; }
            smw = (double)Smw - (double)Cmw;
            smdw = (double)Smdw - (double)Cmdw;
            nn = n_in - 1;  // the particle itself is in its own buffer (r^2 = 0)
        }
        if (exact_finish) {
            // exact walk at the h reached, iterating further if needed
            for (;;) {
                TppDSums<float> S;
                S.sw = S.cw = S.sdw = S.cdw = S.smw = S.cmw = S.smdw = S.cmdw = 0.f;
                S.nn = 0;
                S.hs = 0;
                S.tests = 0;
                tpp_density_walk<float, HASH>(a, B, p, Xi, h, S);
                ++c_evals;
                c_tests += S.tests;
                smw = (double)S.smw - (double)S.cmw;
                smdw = (double)S.smdw - (double)S.cmdw;
                nn = S.nn;
                const double f = (32.0 / 3.0) * ((double)S.sw - (double)S.cw) - a.n_target;
                if (st || fabs(f) <= a.n_tol) break;
                if (it >= a.max_iter) { st |= ST_NOT_CONVERGED; break; }
                ++it;
                const float N = (32.f / 3.f) * (S.sw - S.cw);
                const float dN = -(32.f / 3.f) * (S.sdw - S.cdw) / h;
                if (!h_update(h, f, N, dN, (float)a.n_target, cap, blo, bhi, dold, st)) break;
            }
        }
        const double hd = (double)h;
        a.h[oi] = h;
        a.rho[oi] = (float)(8.0 / (3.141592653589793 * hd * hd * hd) * smw);
        a.omega[oi] = (float)(smdw != 0.0 ? -3.0 * smw / smdw : 1.0);
        a.n_ngb[oi] = nn;
        a.flags[oi] = (uint8_t)st;
        c_pairs += (unsigned long long)nn;
        c_status |= st;
    }
    c_pairs = warp_sum(c_pairs);
    c_evals = warp_sum(c_evals);
    c_tests = warp_sum(c_tests);
    c_status = __reduce_or_sync(0xffffffffu, c_status);
    if (lane_id() == 0) {
        atomicAdd(&a.ctr->density_pairs, c_pairs);
        atomicAdd(&a.ctr->density_evals, c_evals);
        atomicAdd(&a.ctr->pair_tests, c_tests);
        if (c_status) atomicOr(&a.ctr->status, c_status);
    }
}

// ---------------------------------------------------------------------------
// Force
// ---------------------------------------------------------------------------

// Per-call packed records in sorted order: (v, h), (rho, A, c, 1/h), the
// leaf-relative position with h, and (v, m).
__global__ void k_force_pack(int n, const int32_t* __restrict__ perm, const float* __restrict__ vel,
                             const float* __restrict__ u, const float* __restrict__ h, const float* __restrict__ rho,
                             const float* __restrict__ omega, float gam, const float4* __restrict__ posf,
                             float4* __restrict__ fvel, float4* __restrict__ fthermo, float4* __restrict__ fposh,
                             float4* __restrict__ fvm, const uint4* __restrict__ list_xh, unsigned* h_changed,
                             const float* __restrict__ divv, const float* __restrict__ curlv,
                             float* __restrict__ fbal, const float* __restrict__ kappa, float2* __restrict__ fcond,
                             const float* __restrict__ alpha_v, float2* __restrict__ fvisc) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int o = perm[p];
    const float hh = h[o], r = rho[o];
    const float P = (gam - 1.f) * r * u[o];
    const float4 f = posf[p];
    const float vx = vel[3 * (size_t)o], vy = vel[3 * (size_t)o + 1], vz = vel[3 * (size_t)o + 2];
    fvel[p] = make_float4(vx, vy, vz, hh);
    fvm[p] = make_float4(vx, vy, vz, f.w);
    const float cs = sqrtf(gam * P / r);
    fthermo[p] = make_float4(r, omega[o] * P / (r * r), cs, 1.f / hh);
    // Balsara's limiter f = |div v| / (|div v| + |curl v| + 1e-4 c/h)
    float fb = 1.f;
    if (divv) {
        const float ad = fabsf(divv[o]);
        fb = ad / (ad + curlv[o] + 1e-4f * cs / hh);
    }
    if (fbal) fbal[p] = fb;
    if (fvisc) fvisc[p] = make_float2(fb, alpha_v[o]);
    if (fcond) fcond[p] = make_float2(u[o], kappa[o]);
    fposh[p] = make_float4(f.x, f.y, f.z, hh);
    // recorded neighbour lists are usable only if every h equals the one they were made with
    if (list_xh && !(hh == __uint_as_float(list_xh[p].w))) atomicOr(h_changed, 1u);
}

struct TppForceArgs {
    const BoxDesc* boxes;
    int n_boxes;
    const int32_t* act;
    const int* count_ptr;
    int count;
    const uint4* posm;
    const float4* posf;
    const int32_t* perm;
    const uint4* node_c;
    const float4* node_e;
    const float4* fvel;
    const float4* fthermo;
    const float* u;
    const float* omega;
    float* acc;
    float* dudt;
    float* vsig;
    unsigned long long* hash;
    double alpha, gamma;
    Counters* ctr;
};

template <typename T, bool HASH>
__global__ void __launch_bounds__(kTppThreads) k_force_tpp(TppForceArgs a) {
    const int cnt = a.count_ptr ? *a.count_ptr : a.count;
    const T alpha = (T)a.alpha, gam = (T)a.gamma, gm1 = (T)(a.gamma - 1.0);
    const T kNorm = (T)(8.0 / 3.141592653589793);
    unsigned long long c_pairs = 0, c_tests = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
        const int p = a.act[t];
        const BoxDesc& B = a.boxes[a.n_boxes == 1 ? 0 : tpp_box_of(a.boxes, a.n_boxes, p)];
        const double L = B.L, s = ldexp(L, -32);
        const float sf = (float)s;
        const T sT = (T)s;
        const uint4 Xi = a.posm[p];
        const int oi = a.perm[p];
        const float4 vi = a.fvel[p];
        const float4 thi = a.fthermo[p];
        const T hi = (T)vi.w, hinvi = T(1) / hi, rhoi = (T)thi.x;
        T Ai, ci;
        if constexpr (std::is_same<T, float>::value) {
            Ai = thi.y;
            ci = thi.z;
        } else {
            const T Pi = gm1 * rhoi * (T)a.u[oi];
            Ai = (T)a.omega[oi] * Pi / (rhoi * rhoi);
            ci = sqrt(gam * Pi / rhoi);
        }
        const T normi = kNorm * hinvi * hinvi * hinvi * hinvi;
        const double Hd = (double)vi.w * 4294967296.0 / L;
        const double HHi = Hd * Hd;
        const T vxi = (T)vi.x, vyi = (T)vi.y, vzi = (T)vi.z;
        T Sx = 0, Cx = 0, Sy = 0, Cy = 0, Sz = 0, Cz = 0, vsmax = 0;
        double du = 0.0;
        int np = 0;
        unsigned long long hs = 0, tests = 0;

        int stack[kTppStack];
        int sp = 0;
        stack[sp++] = B.nlev == 1 ? 0 : (B.nlev - 1) << 27;
        const long long pend = B.off + B.n;
        while (sp > 0) {
            const int enc = stack[--sp];
            const int lev = enc >> 27, tt = enc & ((1 << 27) - 1);
            if (lev > 0) {
                const int cl = lev - 1;
                const int c0 = tt * kFan, c1 = min(c0 + kFan, B.lvl_n[cl]);
                const int base = B.lvl_off[cl];
                for (int c = c0; c < c1; ++c) {
                    const float4 e = a.node_e[base + c];
                    if (tpp_node_near(a.node_c[base + c], e, Xi, sf, fmaxf(vi.w, e.w))) stack[sp++] = (cl << 27) | c;
                }
                continue;
            }
            const int nd = B.lvl_off[0] + tt;
            const uint4 C = a.node_c[nd];
            const float4 E = a.node_e[nd];
            const T ox = (T)(int)(C.x - Xi.x) * sT, oy = (T)(int)(C.y - Xi.y) * sT, oz = (T)(int)(C.z - Xi.z) * sT;
            const T eL = TBand<T>::rel * (T(4) * (T)(E.x + E.y + E.z) + T(2) * (fabs(ox) + fabs(oy) + fabs(oz)));
            const T elo = T(1) - T(4) * TBand<T>::rel, ehi = T(1) + T(4) * TBand<T>::rel;
            const T ei = eL + TBand<T>::rel * T(2) * hi;
            const T lo2i = hi > ei ? (hi - ei) * (hi - ei) * elo : T(0);
            const T hi2i = (hi + ei) * (hi + ei) * ehi;
            const long long q0 = B.off + (long long)tt * kLeaf, q1 = min(q0 + kLeaf, pend);
            // leaves wider than the minimum-image sum allows: exact integer separations
            const bool wide = T(2) * (T)(E.x + E.y + E.z) + max(hi, (T)E.w) >= T(0.45) * (T)B.L;
            T pax = 0, pay = 0, paz = 0, pdu = 0;
            for (long long q = q0; q < q1; ++q) {
                if (q == p) continue;
                T dx, dy, dz, mj;   // d = x_j - x_i
                if (std::is_same<T, float>::value && !wide) {
                    const float4 f = a.posf[q];
                    dx = ox + f.x; dy = oy + f.y; dz = oz + f.z; mj = f.w;
                } else {
                    const uint4 Xj = a.posm[q];
                    dx = (T)(int)(Xj.x - Xi.x) * sT; dy = (T)(int)(Xj.y - Xi.y) * sT; dz = (T)(int)(Xj.z - Xi.z) * sT;
                    mj = (T)__uint_as_float(Xj.w);
                }
                const T r2 = dx * dx + dy * dy + dz * dz;
                const float4 vj = a.fvel[q];
                const T hj = (T)vj.w;
                const T ej = eL + TBand<T>::rel * T(2) * hj;
                const T hi2j = (hj + ej) * (hj + ej) * ehi;
                const bool mi = r2 < hi2i, mjb = r2 < hi2j;
                if (!(mi || mjb)) continue;
                bool in = r2 < lo2i || r2 < (hj > ej ? (hj - ej) * (hj - ej) * elo : T(0));
                if (!in) {
                    const unsigned long long D2 = exact_d2(Xi, a.posm[q]);
                    const double Hj = (double)vj.w * 4294967296.0 / L;
                    in = (mi && exact_pred(D2, HHi)) || (mjb && exact_pred(D2, Hj * Hj));
                }
                if (!in) continue;
                ++np;
                if (HASH) hs += splitmix64((unsigned long long)a.perm[q]);
                const float4 thj = a.fthermo[q];
                T Aj, cj, hinvj;
                const T rhoj = (T)thj.x;
                if constexpr (std::is_same<T, float>::value) {
                    Aj = thj.y; cj = thj.z; hinvj = thj.w;
                } else {
                    const int o = a.perm[q];
                    const T Pj = gm1 * rhoj * (T)a.u[o];
                    Aj = (T)a.omega[o] * Pj / (rhoj * rhoj);
                    cj = sqrt(gam * Pj / rhoj);
                    hinvj = T(1) / hj;
                }
                if (r2 <= T(0)) {  // coincident: no direction, no force
                    vsmax = max(vsmax, ci + cj);
                    continue;
                }
                T rinv;
                if constexpr (std::is_same<T, float>::value) rinv = rsqrtf(r2);
                else rinv = 1.0 / sqrt(r2);
                const T r = r2 * rinv;
                T w_, dwi, dwj;
                spline<T>(r * hinvi, w_, dwi);
                spline<T>(r * hinvj, w_, dwj);
                const T Fi = normi * dwi * rinv;
                const T Fj = kNorm * hinvj * hinvj * hinvj * hinvj * dwj * rinv;
                // r_ij = x_i - x_j = -d ; v_ij = v_i - v_j
                const T vr = -((vxi - (T)vj.x) * dx + (vyi - (T)vj.y) * dy + (vzi - (T)vj.z) * dz);
                const T wij = vr * rinv;
                const T vs = ci + cj - T(3) * wij;
                vsmax = max(vsmax, vs);
                const T PI = wij < T(0) ? -alpha * vs * wij / (rhoi + rhoj) : T(0);
                const T Fbar = T(0.5) * (Fi + Fj);
                const T coef = mj * (Ai * Fi + Aj * Fj + PI * Fbar);
                pax += coef * dx;   // -coef * r_ij
                pay += coef * dy;
                paz += coef * dz;
                pdu += mj * vr * (Ai * Fi + T(0.5) * PI * Fbar);
            }
            tests += (unsigned long long)(q1 - q0);
            kahan_add(Sx, Cx, pax);
            kahan_add(Sy, Cy, pay);
            kahan_add(Sz, Cz, paz);
            du += (double)pdu;
        }
        a.acc[3 * (size_t)oi] = (float)((double)Sx - (double)Cx);
        a.acc[3 * (size_t)oi + 1] = (float)((double)Sy - (double)Cy);
        a.acc[3 * (size_t)oi + 2] = (float)((double)Sz - (double)Cz);
        a.dudt[oi] = (float)du;
        a.vsig[oi] = (float)vsmax;
        if (HASH) a.hash[oi] = hs;
        c_pairs += (unsigned long long)np;
        c_tests += tests;
    }
    c_pairs = warp_sum(c_pairs);
    c_tests = warp_sum(c_tests);
    if (lane_id() == 0) {
        atomicAdd(&a.ctr->force_pairs, c_pairs);
        atomicAdd(&a.ctr->pair_tests, c_tests);
    }
}

// FP32 force (default): while-while walk; per leaf a cheap membership pass
// builds a bit mask of the pairs in the symmetric set, then the expensive
// pair terms run over the set bits only, so lanes whose leaf has few pairs
// are not dragged through eight evaluations.
template <bool HASH>
__global__ void __launch_bounds__(kTppThreads) k_force_mask(TppForceArgs a) {
    const int cnt = a.count_ptr ? *a.count_ptr : a.count;
    const float alpha = (float)a.alpha;
    const float kNorm = (float)(8.0 / 3.141592653589793);
    const float rel = 9.5367431640625e-07f;  // 2^-20
    const float elo = 1.f - 4.f * rel, ehi = 1.f + 4.f * rel;
    unsigned long long c_pairs = 0, c_tests = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
        const int p = a.act[t];
        const BoxDesc& B = a.boxes[a.n_boxes == 1 ? 0 : tpp_box_of(a.boxes, a.n_boxes, p)];
        const double L = B.L, s = ldexp(L, -32);
        const float sf = (float)s;
        const uint4 Xi = a.posm[p];
        const int oi = a.perm[p];
        const float4 vi = a.fvel[p];
        const float4 thi = a.fthermo[p];
        const float hi = vi.w, hinvi = thi.w, rhoi = thi.x, Ai = thi.y, ci = thi.z;
        const float normi = kNorm * hinvi * hinvi * hinvi * hinvi;
        float Sx = 0.f, Cx = 0.f, Sy = 0.f, Cy = 0.f, Sz = 0.f, Cz = 0.f, Su = 0.f, Cu = 0.f, vsmax = 0.f;
        double HHi = -1.0;  // (h_i 2^32/L)^2, formed on the first band pair only
        int np = 0;
        unsigned long long hs = 0, tests = 0;
        tpp_walk_leaves(B, a.node_c, a.node_e, Xi, sf, hi, true, [&](int lt) {
            const int nd = B.lvl_off[0] + lt;
            const uint4 C = a.node_c[nd];
            const float4 E = a.node_e[nd];
            const long long q0 = B.off + (long long)lt * kLeaf, q1 = min(q0 + kLeaf, B.off + B.n);
            const bool wide = 2.f * (E.x + E.y + E.z) + fmaxf(hi, E.w) >= 0.45f * (float)B.L;
            const float ox = (float)(int)(C.x - Xi.x) * sf, oy = (float)(int)(C.y - Xi.y) * sf,
                        oz = (float)(int)(C.z - Xi.z) * sf;
            const float eL = rel * (4.f * (E.x + E.y + E.z) + 2.f * (fabsf(ox) + fabsf(oy) + fabsf(oz)));
            const float ei = eL + 2.f * rel * hi;
            const float lo2i = hi > ei ? (hi - ei) * (hi - ei) * elo : 0.f;
            const float hi2i = (hi + ei) * (hi + ei) * ehi;
            auto sep = [&](long long q, float& dx, float& dy, float& dz, float& m) {
                if (!wide) {
                    const float4 f = a.posf[q];
                    dx = ox + f.x; dy = oy + f.y; dz = oz + f.z; m = f.w;
                } else {
                    const uint4 Xj = a.posm[q];
                    dx = (float)(int)(Xj.x - Xi.x) * sf; dy = (float)(int)(Xj.y - Xi.y) * sf;
                    dz = (float)(int)(Xj.z - Xi.z) * sf; m = __uint_as_float(Xj.w);
                }
            };
            // pass 1: membership r < max(h_i, h_j), exact inside the band
            unsigned mask = 0u;
            for (long long q = q0; q < q1; ++q) {
                if (q == p) continue;
                float dx, dy, dz, m;
                sep(q, dx, dy, dz, m);
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
                if (in) mask |= 1u << (unsigned)(q - q0);
            }
            tests += (unsigned long long)(q1 - q0);
            // pass 2: pair terms over the members
            float pax = 0.f, pay = 0.f, paz = 0.f, pdu = 0.f;
            while (mask) {
                const int k = __ffs(mask) - 1;
                mask &= mask - 1u;
                const long long q = q0 + k;
                float dx, dy, dz, mj;
                sep(q, dx, dy, dz, mj);
                const float r2 = dx * dx + dy * dy + dz * dz;
                const float4 vj = a.fvel[q];
                const float4 thj = a.fthermo[q];
                ++np;
                if (HASH) hs += splitmix64((unsigned long long)a.perm[q]);
                if (r2 <= 0.f) {  // coincident: no direction, no force
                    vsmax = fmaxf(vsmax, ci + thj.z);
                    continue;
                }
                const float rinv = rsqrtf(r2);
                const float r = r2 * rinv;
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
        });
        a.acc[3 * (size_t)oi] = (float)((double)Sx - (double)Cx);
        a.acc[3 * (size_t)oi + 1] = (float)((double)Sy - (double)Cy);
        a.acc[3 * (size_t)oi + 2] = (float)((double)Sz - (double)Cz);
        a.dudt[oi] = (float)((double)Su - (double)Cu);  // final accumulation in FP64
        a.vsig[oi] = vsmax;
        if (HASH) a.hash[oi] = hs;
        c_pairs += (unsigned long long)np;
        c_tests += tests;
    }
    c_pairs = warp_sum(c_pairs);
    c_tests = warp_sum(c_tests);
    if (lane_id() == 0) {
        atomicAdd(&a.ctr->force_pairs, c_pairs);
        atomicAdd(&a.ctr->pair_tests, c_tests);
    }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------

static int tpp_blocks(sph_ctx* ctx, int bps, int64_t n_active) {
    const long long want = (n_active + kTppThreads - 1) / kTppThreads;
    const long long cap = (long long)ctx->sm_count * (bps > 0 ? bps : 16);
    return (int)std::max<long long>(1, std::min(want, cap));
}

template <typename Kern, typename Args>
static cudaError_t timed_launch(sph_ctx* ctx, Kern k, const Args& args, int blocks, int kind, int timed,
                                cudaStream_t s) {
    cudaEvent_t ea = nullptr, eb = nullptr;
    if (timed) {
        ea = timing_event(ctx);
        eb = timing_event(ctx);
        if (!ea || !eb) return cudaErrorMemoryAllocation;
        cudaEventRecord(ea, s);
    }
    k<<<blocks, kTppThreads, 0, s>>>(args);
    ++ctx->launches;
    if (timed) {
        cudaEventRecord(eb, s);
        ctx->timed.push_back({ea, eb, kind});
    }
    return cudaGetLastError();
}

cudaError_t launch_density_tpp(sph_ctx* ctx, const DensityLaunch& a, int64_t n_active, cudaStream_t s) {
    const sph_grid* g = a.g;
    TppDensArgs da;
    da.boxes = g->boxes;
    da.n_boxes = g->n_boxes;
    da.act = g->act;
    da.count_ptr = reinterpret_cast<const int*>(g->scan + g->n);
    da.count = (int)n_active;
    da.posm = g->posm;
    da.posf = g->posf;
    da.perm = g->perm;
    da.node_c = g->node_c;
    da.node_e = g->node_e;
    da.node_lo = g->node_lo;
    da.node_hi = g->node_hi;
    da.h = a.h;
    da.rho = a.rho;
    da.omega = a.omega;
    da.n_ngb = a.n_ngb;
    da.flags = a.flags;
    da.hash = a.hash;
    da.n_target = a.n_target;
    da.n_tol = a.n_tol;
    da.max_iter = a.max_iter;
    da.fixed_h = a.fixed_h;
    da.guess_h = a.guess_h;
    da.ctr = ctx->counters;
    const int blocks = tpp_blocks(ctx, a.blocks_per_sm, n_active);
    if (a.fp64)
        return a.hash ? timed_launch(ctx, k_density_tpp<double, true>, da, blocks, 0, a.time_kernels, s)
                      : timed_launch(ctx, k_density_tpp<double, false>, da, blocks, 0, a.time_kernels, s);
    if (a.hash || a.fixed_h || !a.buffered)
        return a.hash ? timed_launch(ctx, k_density_tpp<float, true>, da, blocks, 0, a.time_kernels, s)
                      : timed_launch(ctx, k_density_tpp<float, false>, da, blocks, 0, a.time_kernels, s);
    return timed_launch(ctx, k_density_buf<false>, da, blocks, 0, a.time_kernels, s);
}

void force_pack(const sph_grid* g, const float* vel, const float* u, const float* h, const float* rho,
                const float* omega, float gamma, cudaStream_t s, const uint4* list_xh, unsigned* h_changed,
                const float* divv, const float* curlv, const float* kappa, const float* alpha_v) {
    const int n = (int)g->n;
    k_force_pack<<<(n + 255) / 256, 256, 0, s>>>(n, g->perm, vel, u, h, rho, omega, gamma, g->posf, g->fvel, g->fthermo,
                                                 g->fposh, g->fvm, list_xh, h_changed, divv, curlv,
                                                 divv && !alpha_v ? g->fbal : nullptr, kappa,
                                                 kappa ? g->fcond : nullptr, alpha_v,
                                                 alpha_v ? g->fvisc : nullptr);
}

cudaError_t launch_force_tpp(sph_ctx* ctx, const ForceLaunch& a, int64_t n_active, cudaStream_t s) {
    const sph_grid* g = a.g;
    force_pack(g, a.vel, a.u, a.h, a.rho, a.omega, (float)a.gamma, s);
    ++ctx->launches;
    TppForceArgs fa;
    fa.boxes = g->boxes;
    fa.n_boxes = g->n_boxes;
    fa.act = g->act;
    fa.count_ptr = reinterpret_cast<const int*>(g->scan + g->n);
    fa.count = (int)n_active;
    fa.posm = g->posm;
    fa.posf = g->posf;
    fa.perm = g->perm;
    fa.node_c = g->node_c;
    fa.node_e = g->node_e;
    fa.fvel = g->fvel;
    fa.fthermo = g->fthermo;
    fa.u = a.u;
    fa.omega = a.omega;
    fa.acc = a.acc;
    fa.dudt = a.dudt;
    fa.vsig = a.vsig;
    fa.hash = a.hash;
    fa.alpha = a.alpha;
    fa.gamma = a.gamma;
    fa.ctr = ctx->counters;
    const int blocks = tpp_blocks(ctx, a.blocks_per_sm, n_active);
    if (a.fp64)
        return a.hash ? timed_launch(ctx, k_force_tpp<double, true>, fa, blocks, 1, a.time_kernels, s)
                      : timed_launch(ctx, k_force_tpp<double, false>, fa, blocks, 1, a.time_kernels, s);
    return a.hash ? timed_launch(ctx, k_force_mask<true>, fa, blocks, 1, a.time_kernels, s)
                  : timed_launch(ctx, k_force_mask<false>, fa, blocks, 1, a.time_kernels, s);
}

}  // namespace sph
