// force.cu -- SPH hydrodynamic-force pass (the paper's second SPH module,
// Sec. 1), grad-h Gadget-2 form in specific internal energy:
//   a_i    = -sum_j m_j [A_i F_ij(h_i) + A_j F_ij(h_j) + Pi_ij Fbar_ij] r_ij
//   du_i   =  sum_j m_j v_ij.r_ij [A_i F_ij(h_i) + 1/2 Pi_ij Fbar_ij]
// with F_ij(h) = W'(r_ij, h)/r_ij (so grad_i W = F r_ij), Fbar the mean of the
// two, A = Omega P / rho^2, P = (gamma-1) rho u, and the signal-velocity
// viscosity Pi_ij = -(alpha/2) v_sig w_ij / rho_bar for approaching pairs.
// The pair set is symmetric: j != i with r_ij < max(h_i, h_j), so the walk
// radius of a node is max(group h_max, node h_max).
//
//   k_force<T>     one warp per group, the same hierarchy walk as the density
//                  pass (radius widened by the nodes' h_max), candidates staged
//                  in shared memory with everything the pair term needs;
//                  FP32 terms with per-batch Kahan compensation of a, per-batch
//                  FP64 accumulation of du/dt. T = double: all in FP64.
//   k_force_plain  plain FP32 baseline: thread per particle, depth-first walk,
//                  plain FP32 sums.
#include "internal.cuh"
#include "walk.cuh"

namespace sph {

constexpr int kForceWarps = 4;
constexpr int kFCandQ = 64;

template <typename T>
struct FBand;
template <>
struct FBand<float> {
    static constexpr float rel = 9.5367431640625e-07f;  // 2^-20
};
template <>
struct FBand<double> {
    static constexpr double rel = 1.7763568394002505e-15;  // 2^-49
};

__device__ __forceinline__ void fpack_u32(float& d, unsigned v) { d = __uint_as_float(v); }
__device__ __forceinline__ void fpack_u32(double& d, unsigned v) { d = __longlong_as_double((long long)v); }
__device__ __forceinline__ unsigned funpack_u32(float d) { return __float_as_uint(d); }
__device__ __forceinline__ unsigned funpack_u32(double d) { return (unsigned)__double_as_longlong(d); }

template <typename T>
struct alignas(16) FRec {
    T x, y, z, hinv;      // position relative to the group centre (or raw ints), 1/h_j
    T vx, vy, vz, m;
    T rho, A, c, norm;    // rho_j, A_j, c_j, 8/(pi h_j^4)
    T lo2, hi2, h, pad;   // predicate band of h_j, h_j
};

template <typename T>
struct ForceSmem {
    int stack[kStack];
    int leafq[kLeafQ];
    FRec<T> cand[kFCandQ];
    int candj[kFCandQ];
};

struct ForceArgs {
    const BoxDesc* boxes;
    const Group* groups;
    const int* n_groups;
    unsigned* queue;
    const int32_t* act;
    const uint4* posm;
    const int32_t* perm;
    const uint4* node_lo;
    const uint4* node_hi;
    const float* node_hmax;
    const float* vel;
    const float* u;
    const float* h;
    const float* rho;
    const float* omega;
    float* acc;
    float* dudt;
    float* vsig;
    unsigned long long* hash;
    double alpha, gamma;
    Counters* ctr;
};

template <typename T>
__device__ __forceinline__ T rsqrt_t(T x);
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return 1.0 / sqrt(x); }

template <typename T, bool HASH>
__global__ void __launch_bounds__(kForceWarps * 32) k_force(ForceArgs a) {
    __shared__ ForceSmem<T> smem[kForceWarps];
    ForceSmem<T>& sm = smem[threadIdx.x >> 5];
    const unsigned lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    const int ng = *a.n_groups;
    const T gam = (T)a.gamma, gm1 = (T)(a.gamma - 1.0), alpha = (T)a.alpha;
    const T kNorm = (T)(8.0 / 3.141592653589793);
    unsigned long long c_pairs = 0, c_tests = 0, c_groups = 0;

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
        const float hf = valid ? a.h[oi] : 0.f;

        GroupBox gb;
        group_box(Xi, valid, s, gb);
        const float hg = warp_max(hf);
        const T xi = (T)(int)(Xi.x - gb.R[0]) * sT;
        const T yi = (T)(int)(Xi.y - gb.R[1]) * sT;
        const T zi = (T)(int)(Xi.z - gb.R[2]) * sT;
        T vxi = 0, vyi = 0, vzi = 0, rhoi = 1, Ai = 0, ci = 0, hinvi = 0, normi = 0;
        if (valid) {
            vxi = (T)a.vel[3 * (size_t)oi];
            vyi = (T)a.vel[3 * (size_t)oi + 1];
            vzi = (T)a.vel[3 * (size_t)oi + 2];
            rhoi = (T)a.rho[oi];
            const T Pi = gm1 * rhoi * (T)a.u[oi];
            Ai = (T)a.omega[oi] * Pi / (rhoi * rhoi);
            ci = sqrt(gam * Pi / rhoi);
            hinvi = T(1) / (T)hf;
            normi = kNorm * hinvi * hinvi * hinvi * hinvi;
        }
        const T hT = (T)hf;
        const T e = FBand<T>::rel * (T(2) * (T)gb.Emax + T(2) * hT);
        const T lo2 = valid ? (hT > e ? (hT - e) * (hT - e) * (T(1) - T(4) * FBand<T>::rel) : T(0)) : T(-1);
        const T hi2 = valid ? (hT + e) * (hT + e) * (T(1) + T(4) * FBand<T>::rel) : T(-1);
        const double Hd = (double)hf * 4294967296.0 / L;
        const double HHi = Hd * Hd;
        const bool wide = 2.0 * (double)gb.Emax + (double)hg >= 0.45 * L;
        const double to_int = 4294967296.0 / L;
        const float slack = 9.5367431640625e-07f * gb.Emax + 4.f * (float)s;

        T Sx = 0, Cx = 0, Sy = 0, Cy = 0, Sz = 0, Cz = 0;
        double du = 0.0;
        T vsmax = 0;
        int npair = 0;
        unsigned long long hs = 0;
        int nc = 0;

        auto process = [&](int cnt) {
            T pax = 0, pay = 0, paz = 0, pdu = 0;
            for (int k = 0; k < cnt; ++k) {
                const FRec<T>& c = sm.cand[k];
                const int j = sm.candj[k];
                T dx, dy, dz;
                if (wide) {
                    dx = (T)(int)(Xi.x - funpack_u32(c.x)) * sT;
                    dy = (T)(int)(Xi.y - funpack_u32(c.y)) * sT;
                    dz = (T)(int)(Xi.z - funpack_u32(c.z)) * sT;
                } else {
                    dx = xi - c.x;
                    dy = yi - c.y;
                    dz = zi - c.z;
                }
                const T r2 = dx * dx + dy * dy + dz * dz;
                const bool mi = r2 < hi2, mj = r2 < c.hi2;
                if (valid && (mi || mj) && j != p) {
                    bool in = r2 < lo2 || r2 < c.lo2;
                    if (!in) {
                        const unsigned long long D2 = exact_d2(Xi, a.posm[j]);
                        const double Hj = (double)c.h * 4294967296.0 / L;  // same rounding as H_i
                        in = (mi && exact_pred(D2, HHi)) || (mj && exact_pred(D2, Hj * Hj));
                    }
                    if (in) {
                        ++npair;
                        if (HASH) hs += splitmix64((unsigned long long)a.perm[j]);
                        if (r2 > T(0)) {
                            const T rinv = rsqrt_t<T>(r2);
                            const T r = r2 * rinv;
                            T w_, dwi, dwj;
                            spline<T>(r * hinvi, w_, dwi);
                            spline<T>(r * c.hinv, w_, dwj);
                            const T Fi = normi * dwi * rinv;
                            const T Fj = c.norm * dwj * rinv;
                            const T vx = vxi - c.vx, vy = vyi - c.vy, vz = vzi - c.vz;
                            const T vr = vx * dx + vy * dy + vz * dz;
                            const T wij = vr * rinv;
                            const T vs = ci + c.c - T(3) * wij;
                            vsmax = max(vsmax, vs);
                            const T PI = wij < T(0) ? -alpha * vs * wij / (rhoi + c.rho) : T(0);
                            const T Fbar = T(0.5) * (Fi + Fj);
                            const T coef = c.m * (Ai * Fi + c.A * Fj + PI * Fbar);
                            pax -= coef * dx;
                            pay -= coef * dy;
                            paz -= coef * dz;
                            pdu += c.m * vr * (Ai * Fi + T(0.5) * PI * Fbar);
                        } else {
                            vsmax = max(vsmax, ci + c.c);
                        }
                    }
                }
            }
            kahan_add(Sx, Cx, pax);
            kahan_add(Sy, Cy, pay);
            kahan_add(Sz, Cz, paz);
            du += (double)pdu;
            if (valid) c_tests += (unsigned long long)cnt;
        };

        auto test = [&](int lev, int node) -> bool {
            const float r = fmaxf(hg, a.node_hmax[node]);
            const float Rint = (float)((double)r * to_int) * (1.f + 1.5e-5f) + 8.f;
            return node_near(gb, a.node_lo[node], a.node_hi[node], Rint);
        };

        auto tile = [&](int pj) {
            bool pass = false;
            FRec<T> rec;
            if (pj >= 0) {
                const uint4 X = a.posm[pj];
                const int o = a.perm[pj];
                const float hj = a.h[o];
                const T rj = (T)a.rho[o];
                const T Pj = gm1 * rj * (T)a.u[o];
                rec.m = (T)__uint_as_float(X.w);
                rec.h = (T)hj;
                rec.hinv = T(1) / rec.h;
                rec.norm = kNorm * rec.hinv * rec.hinv * rec.hinv * rec.hinv;
                rec.rho = rj;
                rec.A = (T)a.omega[o] * Pj / (rj * rj);
                rec.c = sqrt(gam * Pj / rj);
                rec.vx = (T)a.vel[3 * (size_t)o];
                rec.vy = (T)a.vel[3 * (size_t)o + 1];
                rec.vz = (T)a.vel[3 * (size_t)o + 2];
                const T ej = FBand<T>::rel * (T(2) * (T)gb.Emax + T(2) * rec.h);
                rec.lo2 = rec.h > ej ? (rec.h - ej) * (rec.h - ej) * (T(1) - T(4) * FBand<T>::rel) : T(0);
                rec.hi2 = (rec.h + ej) * (rec.h + ej) * (T(1) + T(4) * FBand<T>::rel);
                rec.pad = 0;
                if (wide) {
                    fpack_u32(rec.x, X.x);
                    fpack_u32(rec.y, X.y);
                    fpack_u32(rec.z, X.z);
                    pass = true;
                } else {
                    rec.x = (T)(int)(X.x - gb.R[0]) * sT;
                    rec.y = (T)(int)(X.y - gb.R[1]) * sT;
                    rec.z = (T)(int)(X.z - gb.R[2]) * sT;
                    const float gx = fmaxf(fabsf((float)rec.x) - gb.E[0], 0.f);
                    const float gy = fmaxf(fabsf((float)rec.y) - gb.E[1], 0.f);
                    const float gz = fmaxf(fabsf((float)rec.z) - gb.E[2], 0.f);
                    const float R = fmaxf(hg, hj) * (1.f + 9.5367431640625e-07f) + slack;
                    pass = gx * gx + gy * gy + gz * gz < R * R;
                }
            }
            const unsigned mk = __ballot_sync(0xffffffffu, pass);
            if (pass) {
                const int slot = nc + __popc(mk & lt);
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

        if (valid) {
            a.acc[3 * (size_t)oi] = (float)((double)Sx - (double)Cx);
            a.acc[3 * (size_t)oi + 1] = (float)((double)Sy - (double)Cy);
            a.acc[3 * (size_t)oi + 2] = (float)((double)Sz - (double)Cz);
            a.dudt[oi] = (float)du;
            a.vsig[oi] = (float)vsmax;
            if (HASH) a.hash[oi] = hs;
            c_pairs += (unsigned long long)npair;
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
// Plain FP32 baseline: one thread per active particle.
// ---------------------------------------------------------------------------

struct PlainForceArgs {
    const BoxDesc* boxes;
    int n_boxes;
    const int32_t* act;
    int count;
    const int* count_ptr;   // device count (subset calls), or NULL
    const uint4* posm;
    const int32_t* perm;
    const uint4* node_lo;
    const uint4* node_hi;
    const float* node_hmax;
    const float* vel;
    const float* u;
    const float* h;
    const float* rho;
    const float* omega;
    float* acc;
    float* dudt;
    float* vsig;
    unsigned long long* hash;
    float alpha, gamma;
    Counters* ctr;
};

__device__ __forceinline__ int fbox_of(const BoxDesc* boxes, int nb, long long p) {
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (boxes[mid].off <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_force_plain(PlainForceArgs a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (a.count_ptr ? *a.count_ptr : a.count)) return;
    const int p = a.act[t];
    const BoxDesc& B = a.boxes[fbox_of(a.boxes, a.n_boxes, p)];
    const float sf = (float)ldexp(B.L, -32);
    const float to_int = (float)(4294967296.0 / B.L);
    const uint4 Xi = a.posm[p];
    const int oi = a.perm[p];
    const float hi = a.h[oi], rhoi = a.rho[oi];
    const float vxi = a.vel[3 * (size_t)oi], vyi = a.vel[3 * (size_t)oi + 1], vzi = a.vel[3 * (size_t)oi + 2];
    const float Pi = (a.gamma - 1.f) * rhoi * a.u[oi];
    const float Ai = a.omega[oi] * Pi / (rhoi * rhoi);
    const float ci = sqrtf(a.gamma * Pi / rhoi);
    const float Hi = hi * to_int;
    float ax = 0.f, ay = 0.f, az = 0.f, du = 0.f, vs = 0.f;
    int np = 0;
    unsigned long long hs = 0;
    int stack[96];
    int sp = 0;
    stack[sp++] = B.nlev == 1 ? 0 : (B.nlev - 1) << 27;
    while (sp > 0) {
        const int enc = stack[--sp];
        const int lev = enc >> 27, tt = enc & ((1 << 27) - 1);
        if (lev == 0) {
            const long long p0 = B.off + (long long)tt * kLeaf, p1 = min(p0 + kLeaf, B.off + B.n);
            for (long long q = p0; q < p1; ++q) {
                if (q == p) continue;
                const uint4 Xj = a.posm[q];
                const int o = a.perm[q];
                const float hj = a.h[o];
                const float dx = (float)(int)(Xi.x - Xj.x) * sf, dy = (float)(int)(Xi.y - Xj.y) * sf,
                            dz = (float)(int)(Xi.z - Xj.z) * sf;
                const float r2 = dx * dx + dy * dy + dz * dz;
                if (!(r2 < hi * hi || r2 < hj * hj)) continue;
                ++np;
                if (a.hash) hs += splitmix64((unsigned long long)o);
                const float rhoj = a.rho[o];
                const float Pj = (a.gamma - 1.f) * rhoj * a.u[o];
                const float cj = sqrtf(a.gamma * Pj / rhoj);
                if (r2 == 0.f) { vs = fmaxf(vs, ci + cj); continue; }
                const float Aj = a.omega[o] * Pj / (rhoj * rhoj);
                const float mj = __uint_as_float(Xj.w);
                const float r = sqrtf(r2);
                float w_, dwi, dwj;
                spline<float>(r / hi, w_, dwi);
                spline<float>(r / hj, w_, dwj);
                const float Fi = 8.f / (3.14159265f * hi * hi * hi * hi) * dwi / r;
                const float Fj = 8.f / (3.14159265f * hj * hj * hj * hj) * dwj / r;
                const float vx = vxi - a.vel[3 * (size_t)o], vy = vyi - a.vel[3 * (size_t)o + 1],
                            vz = vzi - a.vel[3 * (size_t)o + 2];
                const float vr = vx * dx + vy * dy + vz * dz;
                const float w = vr / r;
                const float vsg = ci + cj - 3.f * w;
                vs = fmaxf(vs, vsg);
                const float PI = w < 0.f ? -a.alpha * vsg * w / (rhoi + rhoj) : 0.f;
                const float Fb = 0.5f * (Fi + Fj);
                const float coef = mj * (Ai * Fi + Aj * Fj + PI * Fb);
                ax -= coef * dx;
                ay -= coef * dy;
                az -= coef * dz;
                du += mj * vr * (Ai * Fi + 0.5f * PI * Fb);
            }
        } else {
            const int cl = lev - 1;
            const int c0 = tt * kFan, c1 = min(c0 + kFan, B.lvl_n[cl]);
            for (int c = c0; c < c1; ++c) {
                const int nd = B.lvl_off[cl] + c;
                const uint4 nlo = a.node_lo[nd], nhi = a.node_hi[nd];
                const float R = fmaxf(Hi, a.node_hmax[nd] * to_int) * (1.f + 1.5e-5f) + 8.f;
                const float gx = periodic_gap(Xi.x, Xi.x, nlo.x, nhi.x);
                const float gy = periodic_gap(Xi.y, Xi.y, nlo.y, nhi.y);
                const float gz = periodic_gap(Xi.z, Xi.z, nlo.z, nhi.z);
                if (gx * gx + gy * gy + gz * gz < R * R) stack[sp++] = (cl << 27) | c;
            }
        }
    }
    a.acc[3 * (size_t)oi] = ax;
    a.acc[3 * (size_t)oi + 1] = ay;
    a.acc[3 * (size_t)oi + 2] = az;
    a.dudt[oi] = du;
    a.vsig[oi] = vs;
    if (a.hash) a.hash[oi] = hs;
    atomicAdd(&a.ctr->force_pairs, (unsigned long long)np);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------

template <typename T, bool HASH>
static cudaError_t flaunch_t(sph_ctx* ctx, const ForceArgs& fa, int bps, int timed, cudaStream_t s) {
    int blocks = ctx->sm_count * (bps > 0 ? bps : 4);
    cudaEvent_t ea = nullptr, eb = nullptr;
    if (timed) {
        ea = timing_event(ctx);
        eb = timing_event(ctx);
        if (!ea || !eb) return cudaErrorMemoryAllocation;
        cudaEventRecord(ea, s);
    }
    k_force<T, HASH><<<blocks, kForceWarps * 32, 0, s>>>(fa);
    ++ctx->launches;
    if (timed) {
        cudaEventRecord(eb, s);
        ctx->timed.push_back({ea, eb, 1});
    }
    return cudaGetLastError();
}

static ForceArgs make_args(sph_ctx* ctx, const ForceLaunch& a) {
    const sph_grid* g = a.g;
    ForceArgs fa;
    fa.boxes = g->boxes;
    fa.groups = g->groups;
    fa.n_groups = g->n_groups;
    fa.queue = ctx->queue + 1;
    fa.act = g->act;
    fa.posm = g->posm;
    fa.perm = g->perm;
    fa.node_lo = g->node_lo;
    fa.node_hi = g->node_hi;
    fa.node_hmax = g->node_hmax;
    fa.vel = a.vel;
    fa.u = a.u;
    fa.h = a.h;
    fa.rho = a.rho;
    fa.omega = a.omega;
    fa.acc = a.acc;
    fa.dudt = a.dudt;
    fa.vsig = a.vsig;
    fa.hash = a.hash;
    fa.alpha = a.alpha;
    fa.gamma = a.gamma;
    fa.ctr = ctx->counters;
    return fa;
}

cudaError_t launch_force(sph_ctx* ctx, const ForceLaunch& a, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(ctx->queue + 1, 0, sizeof(unsigned), s);
    if (e) return e;
    ForceArgs fa = make_args(ctx, a);
    const int bps = a.blocks_per_sm, tk = a.time_kernels;
    if (a.fp64)
        return a.hash ? flaunch_t<double, true>(ctx, fa, bps, tk, s) : flaunch_t<double, false>(ctx, fa, bps, tk, s);
    return a.hash ? flaunch_t<float, true>(ctx, fa, bps, tk, s) : flaunch_t<float, false>(ctx, fa, bps, tk, s);
}

cudaError_t launch_force_plain(sph_ctx* ctx, const ForceLaunch& a, int64_t n_active, cudaStream_t s) {
    const sph_grid* g = a.g;
    PlainForceArgs pa;
    pa.boxes = g->boxes;
    pa.n_boxes = g->n_boxes;
    pa.act = g->act;
    pa.count = (int)n_active;
    pa.count_ptr = reinterpret_cast<const int*>(g->scan + g->n);
    pa.posm = g->posm;
    pa.perm = g->perm;
    pa.node_lo = g->node_lo;
    pa.node_hi = g->node_hi;
    pa.node_hmax = g->node_hmax;
    pa.vel = a.vel;
    pa.u = a.u;
    pa.h = a.h;
    pa.rho = a.rho;
    pa.omega = a.omega;
    pa.acc = a.acc;
    pa.dudt = a.dudt;
    pa.vsig = a.vsig;
    pa.hash = a.hash;
    pa.alpha = (float)a.alpha;
    pa.gamma = (float)a.gamma;
    pa.ctr = ctx->counters;
    if (n_active <= 0) return cudaSuccess;
    k_force_plain<<<(int)((n_active + 127) / 128), 128, 0, s>>>(pa);
    ++ctx->launches;
    return cudaGetLastError();
}

}  // namespace sph
