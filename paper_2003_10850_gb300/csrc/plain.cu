// plain.cu -- the plain FP32 baseline of the density and force passes, the
// path the default one is measured against (SPH_PLAIN_FP32):
//   k_density_plain  one thread per particle with its own depth-first walk,
//                    plain FP32 sums, FP32 h update, one launch per iteration
//                    driven by the host;
//   k_force_plain    one thread per active particle, its own walk over
//                    r < max(h_i, h_j), plain FP32 sums.
#include "internal.cuh"
#include "walk.cuh"

namespace sph {

// Initial h from the number density of the particle's leaf and leaf-parent
// boxes (the smaller of the two estimates).
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
