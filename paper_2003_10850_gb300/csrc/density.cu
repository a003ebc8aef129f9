// density.cu -- SPH density pass with on-device smoothing-length iteration.
//
// For each active particle i the pass solves N_eff(h_i) = N_t with
// N_eff(h) = (4 pi/3) h^3 sum_j W(r_ij, h) = (32/3) sum_j w(r_ij/h) (self
// included), then reports rho_i = sum_j m_j W(r_ij,h_i), the grad-h factor
// Omega_i and n_ngb,i. The paper's density module iterates until h settles
// (Sec. 1) and processes neighbours in chunks of 32 (Sec. 2.4).
//
// Two implementations:
//   k_density<T>     one warp per group of <= 32 Morton-consecutive active
//                    particles; one hierarchy walk per iteration for the whole
//                    group; candidates staged in shared memory in batches of
//                    32; FP32 pair terms (T = float) with per-batch Kahan
//                    compensation, FP64 Newton/bisection of h on the device,
//                    iterating until every lane of the group has converged.
//                    T = double runs the same algorithm in FP64.
//   k_density_plain  the plain FP32 baseline: one thread per particle with
//                    its own depth-first walk, plain FP32 sums, FP32 h update,
//                    one launch per iteration driven by the host.
#include "internal.cuh"
#include "walk.cuh"

namespace sph {

constexpr int kDensWarps = 4;
constexpr int kCandQ = 64;

template <typename T>
struct Band;
template <>
struct Band<float> {
    static constexpr float rel = 9.5367431640625e-07f;  // 2^-20
};
template <>
struct Band<double> {
    static constexpr double rel = 1.7763568394002505e-15;  // 2^-49
};

// Carry a raw 32-bit integer in a T slot bit-for-bit (no conversion).
__device__ __forceinline__ void pack_u32(float& d, unsigned v) { d = __uint_as_float(v); }
__device__ __forceinline__ void pack_u32(double& d, unsigned v) { d = __longlong_as_double((long long)v); }
__device__ __forceinline__ unsigned unpack_u32(float d) { return __float_as_uint(d); }
__device__ __forceinline__ unsigned unpack_u32(double d) { return (unsigned)__double_as_longlong(d); }

template <typename T>
struct alignas(16) DRec {
    T x, y, z, m;
};

template <typename T>
struct DensSmem {
    int stack[kStack];
    int leafq[kLeafQ];
    DRec<T> cand[kCandQ];
    int candj[kCandQ];
};

struct DensArgs {
    const BoxDesc* boxes;
    const Group* groups;
    const int* n_groups;
    unsigned* queue;
    const int32_t* act;
    const uint4* posm;
    const int32_t* perm;
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
__device__ __forceinline__ T sqrt_t(T x);
template <>
__device__ __forceinline__ float sqrt_t<float>(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }
template <>
__device__ __forceinline__ double sqrt_t<double>(double x) { return sqrt(x); }

// Local starting guess for h: the number density inside the bounding boxes
// of the particle's leaf (8 sorted particles) and of the leaf's parent (64);
// the smaller of the two estimates, since growing h from below is cheap while
// a first evaluation far above the root touches many candidates.
__device__ float guess_h(const BoxDesc& B, const uint4* node_lo, const uint4* node_hi, long long p,
                         double s, double n_target) {
    double best = 0.25 * B.L;
    const int top = B.nlev > 1 ? 1 : 0;
    for (int lev = 0; lev <= top; ++lev) {
        long long span = lev ? (long long)kLeaf * kFan : kLeaf;
        long long t = (p - B.off) / span;
        uint4 lo = node_lo[B.lvl_off[lev] + t], hi = node_hi[B.lvl_off[lev] + t];
        double cnt = (double)min(span, B.n - t * span);
        double V = ((double)(hi.x - lo.x) + 1.0) * ((double)(hi.y - lo.y) + 1.0) *
                   ((double)(hi.z - lo.z) + 1.0) * s * s * s;
        best = fmin(best, cbrt(3.0 * n_target * V / (4.0 * 3.141592653589793 * cnt)));
    }
    return (float)best;
}

template <typename T, bool HASH>
__global__ void __launch_bounds__(kDensWarps * 32) k_density(DensArgs a) {
    __shared__ DensSmem<T> smem[kDensWarps];
    DensSmem<T>& sm = smem[threadIdx.x >> 5];
    const unsigned lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
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
        const double L = B.L;
        const double s = ldexp(L, -32);
        const T sT = (T)s;
        const bool valid = (int)lane < G.count;
        const int p = valid ? a.act[G.first + lane] : -1;
        const uint4 Xi = valid ? a.posm[p] : make_uint4(0, 0, 0, 0);
        const int oi = valid ? a.perm[p] : 0;
        float h = valid ? a.h[oi] : 0.f;
        if (valid && (a.guess_h || !(h > 0.f) || !isfinite(h))) h = guess_h(B, a.node_lo, a.node_hi, p, s, a.n_target);

        GroupBox gb;
        group_box(Xi, valid, s, gb);
        const T xi = (T)(int)(Xi.x - gb.R[0]) * sT;
        const T yi = (T)(int)(Xi.y - gb.R[1]) * sT;
        const T zi = (T)(int)(Xi.z - gb.R[2]) * sT;

        double blo = 0.0, bhi = INFINITY;
        const double cap = 0.5 * L * (1.0 - 1e-9);
        bool conv = !valid;
        unsigned st = 0;
        T Sw = 0, Cw = 0, Sdw = 0, Cdw = 0, Smw = 0, Cmw = 0, Smdw = 0, Cmdw = 0;
        int nn = 0;
        unsigned long long hs = 0;
        int nc = 0;  // candidates staged in sm.cand

        for (int it = 0;; ++it) {
            const float hg = warp_max(conv ? 0.f : h);
            const bool wide = 2.0 * (double)gb.Emax + (double)hg >= 0.45 * L;
            // per-lane predicate thresholds (see exact_pred): r2 < lo2 is a
            // sure neighbour, r2 >= hi2 a sure non-neighbour, in between the
            // exact integer/FP64 test decides.
            T hT = (T)h, hinv = conv ? T(0) : T(1) / hT;
            T e = Band<T>::rel * (T(2) * (T)gb.Emax + T(2) * hT);
            T lo2 = conv ? T(-1) : (hT > e ? (hT - e) * (hT - e) * (T(1) - T(4) * Band<T>::rel) : T(0));
            T hi2 = conv ? T(-1) : (hT + e) * (hT + e) * (T(1) + T(4) * Band<T>::rel);
            double Hd = (double)h * 4294967296.0 / L;
            double HH = Hd * Hd;
            if (!conv) {
                Sw = Cw = Sdw = Cdw = Smw = Cmw = Smdw = Cmdw = 0;
                nn = 0;
                hs = 0;
            }
            const float cullR = (float)hg + 9.5367431640625e-07f * (gb.Emax + (float)hg) + 4.f * (float)s;
            const float cull2 = cullR * cullR;
            const float Rint = (float)((double)hg * 4294967296.0 / L) * (1.f + 1.5e-5f) + 8.f;

            auto process = [&](int cnt) {
                T pw = 0, pdw = 0, pmw = 0, pmdw = 0;
                int pn = 0;
                unsigned long long ph = 0;
                for (int k = 0; k < cnt; ++k) {
                    const DRec<T> c = sm.cand[k];
                    const int j = sm.candj[k];
                    T dx, dy, dz, m;
                    if (wide) {
                        dx = (T)(int)(Xi.x - unpack_u32(c.x)) * sT;
                        dy = (T)(int)(Xi.y - unpack_u32(c.y)) * sT;
                        dz = (T)(int)(Xi.z - unpack_u32(c.z)) * sT;
                    } else {
                        dx = xi - c.x;
                        dy = yi - c.y;
                        dz = zi - c.z;
                    }
                    m = c.m;
                    const T r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 < hi2) {
                        bool in = r2 < lo2;
                        if (!in) in = exact_pred(exact_d2(Xi, a.posm[j]), HH);
                        if (in) {
                            const T q = sqrt_t<T>(r2) * hinv;
                            T w, dw;
                            spline<T>(q, w, dw);
                            const T qdw = q * dw;
                            pw += w;
                            pdw += qdw;
                            pmw += m * w;
                            pmdw += m * qdw;
                            if (j != p) {
                                ++pn;
                                if (HASH) ph += splitmix64((unsigned long long)a.perm[j]);
                            }
                        }
                    }
                }
                if (!conv) {
                    kahan_add(Sw, Cw, pw);
                    kahan_add(Sdw, Cdw, pdw);
                    kahan_add(Smw, Cmw, pmw);
                    kahan_add(Smdw, Cmdw, pmdw);
                    nn += pn;
                    hs += ph;
                    c_tests += (unsigned long long)cnt;
                }
            };

            auto test = [&](int lev, int node) -> bool {
                return node_near(gb, a.node_lo[node], a.node_hi[node], Rint);
            };

            auto tile = [&](int pj) {
                bool pass = false;
                DRec<T> rec;
                rec.x = rec.y = rec.z = rec.m = 0;
                if (pj >= 0) {
                    const uint4 X = a.posm[pj];
                    rec.m = (T)__uint_as_float(X.w);
                    if (wide) {
                        // raw integer coordinates carried in the record
                        pack_u32(rec.x, X.x);
                        pack_u32(rec.y, X.y);
                        pack_u32(rec.z, X.z);
                        pass = true;
                    } else {
                        rec.x = (T)(int)(X.x - gb.R[0]) * sT;
                        rec.y = (T)(int)(X.y - gb.R[1]) * sT;
                        rec.z = (T)(int)(X.z - gb.R[2]) * sT;
                        float gx = fmaxf(fabsf((float)rec.x) - gb.E[0], 0.f);
                        float gy = fmaxf(fabsf((float)rec.y) - gb.E[1], 0.f);
                        float gz = fmaxf(fabsf((float)rec.z) - gb.E[2], 0.f);
                        pass = gx * gx + gy * gy + gz * gz < cull2;
                    }
                }
                const unsigned mk = __ballot_sync(0xffffffffu, pass);
                if (pass) {
                    int slot = nc + __popc(mk & lt);
                    sm.cand[slot] = rec;
                    sm.candj[slot] = pj;
                }
                nc += __popc(mk);
                __syncwarp();
                if (nc >= 32) {
                    process(32);
                    __syncwarp();
                    if ((int)lane < nc - 32) {
                        sm.cand[lane] = sm.cand[lane + 32];
                        sm.candj[lane] = sm.candj[lane + 32];
                    }
                    nc -= 32;
                    __syncwarp();
                }
            };

            walk_box(B, sm.stack, sm.leafq, test, tile);
            if (nc > 0) {
                process(nc);
                nc = 0;
                __syncwarp();
            }

            // FP64 smoothing-length update per unconverged lane
            if (!conv) {
                ++c_evals;
                const double sw = (double)Sw - (double)Cw;
                const double sdw = (double)Sdw - (double)Cdw;
                const double N = (32.0 / 3.0) * sw;
                const double dN = -(32.0 / 3.0) * sdw / (double)h;
                const double f = N - a.n_target;
                if (a.fixed_h || fabs(f) <= a.n_tol) {
                    conv = true;
                } else if (it >= a.max_iter) {
                    conv = true;
                    st |= ST_NOT_CONVERGED;
                } else {
                    if (f < 0) blo = h; else bhi = h;
                    // Newton on N^(1/3) - N_t^(1/3) (nearly linear in h, both for
                    // uniform neighbourhoods, N ~ h^3, and at density fronts,
                    // N ~ (h - r0)^3), kept inside the bracket; grow while
                    // unbracketed; bisect when Newton leaves the bracket.
                    double hn = dN > 0.0 ? (double)h - 3.0 * N * (1.0 - cbrt(a.n_target / N)) / dN : NAN;
                    if (isinf(bhi)) {
                        if ((double)h >= cap) {
                            st |= ST_H_TOO_LARGE;
                            conv = true;
                        } else {
                            if (!(hn > (double)h)) hn = 2.0 * (double)h;
                            hn = fmin(hn, fmin(cap, 8.0 * (double)h));
                        }
                    } else if (!(hn > blo && hn < bhi)) {
                        hn = 0.5 * (blo + bhi);
                    }
                    if (!conv) {
                        float hf = (float)hn;
                        // rounding to float may land on a bracket end: if the
                        // bracket is one float apart, h is the best float there is
                        if (!(hf > (float)blo) || (!isinf(bhi) && !(hf < (float)bhi))) {
                            const float mid = (float)(0.5 * (blo + bhi));
                            hf = (mid > (float)blo && mid < (float)bhi) ? mid : h;
                        }
                        if (hf == h) conv = true;
                        else h = hf;
                    }
                }
            }
            if (__all_sync(0xffffffffu, conv)) break;
        }

        if (valid) {
            const double smw = (double)Smw - (double)Cmw;
            const double smdw = (double)Smdw - (double)Cmdw;
            const double hd = (double)h;
            const double rho = 8.0 / (3.141592653589793 * hd * hd * hd) * smw;
            const double om = smdw != 0.0 ? -3.0 * smw / smdw : 1.0;
            a.h[oi] = h;
            a.rho[oi] = (float)rho;
            a.omega[oi] = (float)om;
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
// Plain FP32 baseline: one thread per particle, one launch per iteration.
// ---------------------------------------------------------------------------

struct PlainDensArgs {
    const BoxDesc* boxes;
    int n_boxes;
    const uint4* posm;
    const int32_t* perm;
    const uint4* node_lo;
    const uint4* node_hi;
    const int32_t* list;
    const int* list_n;   // NULL: use count
    int count;
    int32_t* next;
    int* next_n;
    float* st_lo;
    float* st_hi;
    int first;
    int last;
    float* h;
    float* rho;
    float* omega;
    int32_t* n_ngb;
    uint8_t* flags;
    unsigned long long* hash;
    float n_target, n_tol;
    int fixed_h, guess_h;
    Counters* ctr;
};

__device__ __forceinline__ int box_of(const BoxDesc* boxes, int nb, long long p) {
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (boxes[mid].off <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_density_plain(PlainDensArgs a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int cnt = a.list_n ? *a.list_n : a.count;
    if (t >= cnt) return;
    const int p = a.list[t];
    const BoxDesc& B = a.boxes[box_of(a.boxes, a.n_boxes, p)];
    const float L = (float)B.L;
    const double s = ldexp(B.L, -32);
    const uint4 Xi = a.posm[p];
    const int oi = a.perm[p];
    float h = a.h[oi];
    if (a.first && (a.guess_h || !(h > 0.f) || !isfinite(h))) h = guess_h(B, a.node_lo, a.node_hi, p, s, a.n_target);
    float lo = a.first ? 0.f : a.st_lo[p];
    float hi = a.first ? INFINITY : a.st_hi[p];

    const float Hu = h * (float)(4294967296.0 / B.L);  // h in integer units
    const float H2 = Hu * Hu;
    const float Rint = Hu * (1.f + 1.5e-5f) + 8.f;
    float sw = 0.f, sdw = 0.f, smw = 0.f, smdw = 0.f;
    int nn = 0;
    unsigned long long hs = 0;
    int stack[96];
    int sp = 0;
    if (B.nlev == 1) stack[sp++] = 0;
    else stack[sp++] = (B.nlev - 1) << 27;
    const float invH = 1.f / Hu;
    while (sp > 0) {
        int enc = stack[--sp];
        int lev = enc >> 27, tt = enc & ((1 << 27) - 1);
        if (lev == 0) {
            long long p0 = B.off + (long long)tt * kLeaf, p1 = min(p0 + kLeaf, B.off + B.n);
            for (long long q = p0; q < p1; ++q) {
                uint4 Xj = a.posm[q];
                float dx = (float)(int)(Xi.x - Xj.x), dy = (float)(int)(Xi.y - Xj.y), dz = (float)(int)(Xi.z - Xj.z);
                float r2 = dx * dx + dy * dy + dz * dz;
                if (r2 < H2) {
                    float qq = sqrtf(r2) * invH;
                    float w, dw;
                    spline<float>(qq, w, dw);
                    float m = __uint_as_float(Xj.w);
                    sw += w;
                    sdw += qq * dw;
                    smw += m * w;
                    smdw += m * qq * dw;
                    if (q != p) {
                        ++nn;
                        if (a.hash) hs += splitmix64((unsigned long long)a.perm[q]);
                    }
                }
            }
        } else {
            int cl = lev - 1;
            int c0 = tt * kFan, c1 = min(c0 + kFan, B.lvl_n[cl]);
            for (int c = c0; c < c1; ++c) {
                int nd = B.lvl_off[cl] + c;
                uint4 nlo = a.node_lo[nd], nhi = a.node_hi[nd];
                float gx = periodic_gap(Xi.x, Xi.x, nlo.x, nhi.x);
                float gy = periodic_gap(Xi.y, Xi.y, nlo.y, nhi.y);
                float gz = periodic_gap(Xi.z, Xi.z, nlo.z, nhi.z);
                if (gx * gx + gy * gy + gz * gz < Rint * Rint) stack[sp++] = (cl << 27) | c;
            }
        }
    }
    const float N = (32.f / 3.f) * sw;
    const float dN = -(32.f / 3.f) * sdw / h;
    const float f = N - a.n_target;
    bool done = a.fixed_h || fabsf(f) <= a.n_tol;
    unsigned st = 0;
    if (!done && a.last) { done = true; st |= ST_NOT_CONVERGED; }
    float hn = h;
    if (!done) {
        if (f < 0.f) lo = h; else hi = h;
        hn = dN > 0.f ? h - 3.f * N * (1.f - cbrtf(a.n_target / N)) / dN : NAN;
        if (isinf(hi)) {
            if (h >= 0.499f * L) { st |= ST_H_TOO_LARGE; done = true; }
            if (!(hn > h)) hn = 2.f * h;
            hn = fminf(hn, fminf(0.499f * L, 8.f * h));
        } else if (!(hn > lo && hn < hi)) {
            hn = 0.5f * (lo + hi);
        }
        if (!(hn > lo) || (!isinf(hi) && !(hn < hi)) || hn == h) done = true;  // bracket is one float wide
    }
    if (done) {
        a.h[oi] = h;
        a.rho[oi] = 8.f / (3.14159265f * h * h * h) * smw;
        a.omega[oi] = smdw != 0.f ? -3.f * smw / smdw : 1.f;
        a.n_ngb[oi] = nn;
        a.flags[oi] = (uint8_t)st;
        if (a.hash) a.hash[oi] = hs;
        atomicAdd(&a.ctr->density_pairs, (unsigned long long)nn);
        if (st) atomicOr(&a.ctr->status, st);
    } else {
        a.h[oi] = hn;
        a.st_lo[p] = lo;
        a.st_hi[p] = hi;
        int slot = atomicAdd(a.next_n, 1);
        a.next[slot] = p;
    }
    atomicAdd(&a.ctr->density_evals, 1ull);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------

template <typename T, bool HASH>
static cudaError_t launch_t(sph_ctx* ctx, const DensArgs& da, int bps, int timed, cudaStream_t s) {
    int blocks = ctx->sm_count * (bps > 0 ? bps : 4);
    cudaEvent_t ea = nullptr, eb = nullptr;
    if (timed) {
        ea = timing_event(ctx);
        eb = timing_event(ctx);
        if (!ea || !eb) return cudaErrorMemoryAllocation;
        cudaEventRecord(ea, s);
    }
    k_density<T, HASH><<<blocks, kDensWarps * 32, 0, s>>>(da);
    ++ctx->launches;
    if (timed) {
        cudaEventRecord(eb, s);
        ctx->timed.push_back({ea, eb, 0});
    }
    return cudaGetLastError();
}

cudaError_t launch_density(sph_ctx* ctx, const DensityLaunch& a, cudaStream_t s) {
    const sph_grid* g = a.g;
    cudaError_t e = cudaMemsetAsync(ctx->queue, 0, sizeof(unsigned), s);
    if (e) return e;
    DensArgs da;
    da.boxes = g->boxes;
    da.groups = g->groups;
    da.n_groups = g->n_groups;
    da.queue = ctx->queue;
    da.act = g->act;
    da.posm = g->posm;
    da.perm = g->perm;
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
    const int bps = a.blocks_per_sm, tk = a.time_kernels;
    if (a.fp64)
        return a.hash ? launch_t<double, true>(ctx, da, bps, tk, s) : launch_t<double, false>(ctx, da, bps, tk, s);
    return a.hash ? launch_t<float, true>(ctx, da, bps, tk, s) : launch_t<float, false>(ctx, da, bps, tk, s);
}

cudaError_t run_density_plain(sph_ctx* ctx, const DensityLaunch& a, int64_t n_active, cudaStream_t s) {
    const sph_grid* g = a.g;
    PlainDensArgs pa;
    pa.boxes = g->boxes;
    pa.n_boxes = g->n_boxes;
    pa.posm = g->posm;
    pa.perm = g->perm;
    pa.node_lo = g->node_lo;
    pa.node_hi = g->node_hi;
    pa.st_lo = g->st_lo;
    pa.st_hi = g->st_hi;
    pa.h = a.h;
    pa.rho = a.rho;
    pa.omega = a.omega;
    pa.n_ngb = a.n_ngb;
    pa.flags = a.flags;
    pa.hash = a.hash;
    pa.n_target = (float)a.n_target;
    pa.n_tol = (float)a.n_tol;
    pa.fixed_h = a.fixed_h;
    pa.guess_h = a.guess_h;
    pa.ctr = ctx->counters;
    // the first pass reads the active count from the device (the compacted
    // active list drops duplicates); later passes read it back to decide
    int count = (int)n_active;
    const int* count0 = reinterpret_cast<const int*>(g->scan + g->n);
    const int32_t* list = g->act;
    int32_t* bufs[2] = {g->list_a, g->list_b};
    int which = 0;
    for (int it = 0; count > 0; ++it) {
        cudaError_t e = cudaMemsetAsync(g->list_n + which, 0, sizeof(int), s);
        if (e) return e;
        pa.list = list;
        pa.list_n = it == 0 ? count0 : nullptr;
        pa.count = count;
        pa.next = bufs[which];
        pa.next_n = g->list_n + which;
        pa.first = it == 0;
        pa.last = it >= a.max_iter;
        k_density_plain<<<(count + 127) / 128, 128, 0, s>>>(pa);
        ++ctx->launches;
        if ((e = cudaGetLastError())) return e;
        int next = 0;
        if ((e = cudaMemcpyAsync(&next, g->list_n + which, sizeof(int), cudaMemcpyDeviceToHost, s))) return e;
        if ((e = cudaStreamSynchronize(s))) return e;
        list = bufs[which];
        which ^= 1;
        count = next;
    }
    return cudaSuccess;
}

}  // namespace sph
