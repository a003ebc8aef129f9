// backward.cu -- adjoint of the density and force passes (sph_backward).
//
// Given seeds abar_i = dL/da_i and rhobar_i = dL/drho_i for all particles,
// returns dL/dx, dL/du and dL/dm through the whole forward chain:
//   h_i(x)        implicit: N_i(h_i, x) = N_t (number-weighted, mass-free)
//   rho_i, D_i    = sum_j m_j {W, dW/dh}(r_ij, h_i)
//   Omega_i       = 1 / (1 + h_i D_i / (3 rho_i))
//   a_i           = sum_j m_j G_ij (x_j - x_i),
//   G_ij          = A_i F(r,h_i) + A_j F(r,h_j) + Pi_ij (F(r,h_i)+F(r,h_j))/2,
//   A = Omega (gamma-1) u / rho, c = sqrt(gamma (gamma-1) u), F = W_r / r.
// Reverse mode runs as three gathers over each particle's symmetric pair set
// (j != k, r_kj < max(h_k, h_j)), so every particle collects its own adjoint
// without atomics (deterministic):
//   pass 0  force adjoint: x, m (explicit), and the adjoints of h, A, c, rho;
//           per particle it then folds A, c into u, Omega, rho and the Omega
//           adjoint into h, D, rho;
//   pass 1  density adjoint: x and m through rho and D, h through D, and the
//           implicit-h multiplier lambda_k = hbar_k / (dN_k/dh_k);
//   pass 2  implicit h: x through N, weighted by lambda.
// FP32 pair terms with per-leaf Kahan compensation. The paper has no
// gradients; this is the build's extension of its hot path.
#include <algorithm>

#include "internal.cuh"

namespace sph {

constexpr int kBwThreads = 128;
constexpr int kBwStack = 96;

// w, w', w'' of the cubic spline (branch-free, as spline()).
__device__ __forceinline__ void spline2(float q, float& w, float& dw, float& ddw) {
    const float a = fmaxf(1.f - q, 0.f), b = fmaxf(0.5f - q, 0.f);
    const float a2 = a * a, b2 = b * b;
    w = 2.f * a2 * a - 8.f * b2 * b;
    dw = 24.f * b2 - 6.f * a2;
    ddw = 12.f * a - 48.f * b;
}

__device__ __forceinline__ bool bw_node_near(uint4 c, float4 e, uint4 X, float sf, float R) {
    const float dx = (float)(int)(c.x - X.x) * sf, dy = (float)(int)(c.y - X.y) * sf,
                dz = (float)(int)(c.z - X.z) * sf;
    const float gx = fmaxf(fabsf(dx) - e.x, 0.f), gy = fmaxf(fabsf(dy) - e.y, 0.f),
                gz = fmaxf(fabsf(dz) - e.z, 0.f);
    const float Rt = R * (1.f + 3.0517578125e-05f) + 2.384185791015625e-07f * (fabsf(dx) + fabsf(dy) + fabsf(dz)) +
                     4.f * sf;
    return gx * gx + gy * gy + gz * gz < Rt * Rt;
}

struct BwArgs {
    const BoxDesc* boxes;
    int n_boxes;
    int n;
    const uint4* posm;
    const float4* posf;
    const uint4* node_c;
    const float4* node_e;
    const float4* fvel;     // v, h
    const float4* fthermo;  // rho, A, c, 1/h
    const float4* ga;       // abar (xyz), rhobar seed (w)
    const float* u;         // sorted u
    const float* omega;     // sorted Omega
    float4* xbar;           // accumulated dL/dx (xyz)
    float* mbar;
    float* ubar;
    float* hbar;
    float2* rd;             // total rhobar, Dbar
    float* lam;
    float alpha, gamma;
};

// Sorted copies of the seeds, u and Omega.
__global__ void k_bw_prep(int n, const int32_t* __restrict__ perm, const float* __restrict__ g_acc,
                          const float* __restrict__ g_rho, const float* __restrict__ u,
                          const float* __restrict__ omega, float4* __restrict__ ga, float* __restrict__ us,
                          float* __restrict__ oms) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int o = perm[p];
    ga[p] = make_float4(g_acc[3 * (size_t)o], g_acc[3 * (size_t)o + 1], g_acc[3 * (size_t)o + 2],
                        g_rho ? g_rho[o] : 0.f);
    us[p] = u[o];
    oms[p] = omega[o];
}

__global__ void k_bw_scatter(int n, const int32_t* __restrict__ perm, const float4* __restrict__ xbar,
                             const float* __restrict__ ubar, const float* __restrict__ mbar,
                             float* __restrict__ g_pos, float* __restrict__ g_u, float* __restrict__ g_mass) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int o = perm[p];
    const float4 x = xbar[p];
    g_pos[3 * (size_t)o] = x.x;
    g_pos[3 * (size_t)o + 1] = x.y;
    g_pos[3 * (size_t)o + 2] = x.z;
    g_u[o] = ubar[p];
    g_mass[o] = mbar[p];
}

__device__ __forceinline__ int bw_box_of(const BoxDesc* boxes, int nb, long long p) {
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (boxes[mid].off <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <int PASS>
__global__ void __launch_bounds__(kBwThreads) k_backward(BwArgs a) {
    const float kN = 2.5464790894703255f;  // 8/pi
    const float alpha = a.alpha, gam = a.gamma;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.n; k += gridDim.x * blockDim.x) {
        const BoxDesc& B = a.boxes[a.n_boxes == 1 ? 0 : bw_box_of(a.boxes, a.n_boxes, k)];
        const double s = ldexp(B.L, -32);
        const float sf = (float)s;
        const uint4 Xk = a.posm[k];
        const float mk = __uint_as_float(Xk.w);
        const float4 vk = a.fvel[k];
        const float4 tk = a.fthermo[k];
        const float hk = vk.w, hinvk = tk.w, rhok = tk.x, Ak = tk.y, ck = tk.z;
        const float nk4 = kN * hinvk * hinvk * hinvk * hinvk;   // (8/pi) h^-4
        float4 gk = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 rdk = make_float2(0.f, 0.f);
        float lamk = 0.f;
        if (PASS == 0) gk = a.ga[k];
        if (PASS == 1) rdk = a.rd[k];
        if (PASS == 2) lamk = a.lam[k];
        // accumulators (Kahan per leaf)
        float Sx = 0.f, Cx = 0.f, Sy = 0.f, Cy = 0.f, Sz = 0.f, Cz = 0.f;
        float Sm = 0.f, Cm = 0.f, Sh = 0.f, Ch = 0.f, SA = 0.f, CA = 0.f, Sc = 0.f, Cc = 0.f, Sr = 0.f, Cr = 0.f;
        float SdN = 0.f, CdN = 0.f;

        int stack[kBwStack];
        int sp = 0;
        stack[sp++] = B.nlev == 1 ? 0 : (B.nlev - 1) << 27;
        for (;;) {
            int lt = -1;
            while (sp > 0) {
                const int enc = stack[--sp];
                const int lev = enc >> 27, t = enc & ((1 << 27) - 1);
                if (lev == 0) { lt = t; break; }
                const int cl = lev - 1;
                const int c0 = t * kFan, c1 = min(c0 + kFan, B.lvl_n[cl]);
                const int base = B.lvl_off[cl];
                for (int c = c0; c < c1; ++c) {
                    const float4 e = a.node_e[base + c];
                    if (bw_node_near(a.node_c[base + c], e, Xk, sf, fmaxf(hk, e.w))) stack[sp++] = (cl << 27) | c;
                }
            }
            if (lt < 0) break;
            const int nd = B.lvl_off[0] + lt;
            const uint4 C = a.node_c[nd];
            const float4 E = a.node_e[nd];
            const long long q0 = B.off + (long long)lt * kLeaf, q1 = min(q0 + kLeaf, B.off + B.n);
            const bool wide = 2.f * (E.x + E.y + E.z) + fmaxf(hk, E.w) >= 0.45f * (float)B.L;
            const float ox = (float)(int)(C.x - Xk.x) * sf, oy = (float)(int)(C.y - Xk.y) * sf,
                        oz = (float)(int)(C.z - Xk.z) * sf;
            float px = 0.f, py = 0.f, pz = 0.f, pm = 0.f, ph = 0.f, pA = 0.f, pc = 0.f, pr = 0.f, pdN = 0.f;
            for (long long q = q0; q < q1; ++q) {
                if (q == k) continue;
                float dx, dy, dz, mj;   // d = x_j - x_k
                if (!wide) {
                    const float4 f = a.posf[q];
                    dx = ox + f.x; dy = oy + f.y; dz = oz + f.z; mj = f.w;
                } else {
                    const uint4 Xj = a.posm[q];
                    dx = (float)(int)(Xj.x - Xk.x) * sf; dy = (float)(int)(Xj.y - Xk.y) * sf;
                    dz = (float)(int)(Xj.z - Xk.z) * sf; mj = __uint_as_float(Xj.w);
                }
                const float r2 = dx * dx + dy * dy + dz * dz;
                const float4 vj = a.fvel[q];
                const float hj = vj.w;
                const float hm = fmaxf(hk, hj);
                if (!(r2 < hm * hm) || r2 <= 0.f) continue;
                const float rinv = rsqrtf(r2), r = r2 * rinv;
                const float ux = dx * rinv, uy = dy * rinv, uz = dz * rinv;   // d-hat; e_kj = -d-hat
                const float hinvj = 1.f / hj;
                const float qk = r * hinvk, qj = r * hinvj;
                float wk, dwk, ddwk, wj, dwj, ddwj;
                spline2(qk, wk, dwk, ddwk);
                spline2(qj, wj, dwj, ddwj);
                if (PASS == 0) {
                    const float4 tj = a.fthermo[q];
                    const float4 gj = a.ga[q];
                    const float rhoj = tj.x, Aj = tj.y, cj = tj.z;
                    const float nj4 = kN * hinvj * hinvj * hinvj * hinvj;
                    const float Fk = nk4 * dwk * rinv, Fj = nj4 * dwj * rinv;
                    const float Fbar = 0.5f * (Fk + Fj);
                    // F_r = (8/pi) h^-4 (w''/(h r) - w'/r^2), F_h = -(8/pi) h^-5 (4w' + q w'')/r
                    const float Frk = nk4 * (ddwk * hinvk * rinv - dwk * rinv * rinv);
                    const float Frj = nj4 * (ddwj * hinvj * rinv - dwj * rinv * rinv);
                    const float Fhk = -nk4 * hinvk * (4.f * dwk + qk * ddwk) * rinv;
                    const float vx = vk.x - vj.x, vy = vk.y - vj.y, vz = vk.z - vj.z;   // v_kj
                    const float w = -(vx * ux + vy * uy + vz * uz);                      // v_kj . r_kj / r
                    const float rbar = 0.5f * (rhok + rhoj);
                    const float vsig = ck + cj - 3.f * w;
                    const bool visc = w < 0.f;
                    const float PI = visc ? -0.5f * alpha * vsig * w / rbar : 0.f;
                    const float PIw = visc ? -0.5f * alpha * (vsig - 3.f * w) / rbar : 0.f;
                    const float PIc = visc ? -0.5f * alpha * w / rbar : 0.f;
                    const float PIr = visc ? -0.5f * PI / rbar : 0.f;
                    const float G = Ak * Fk + Aj * Fj + PI * Fbar;
                    const float Gr = (Ak + 0.5f * PI) * Frk + (Aj + 0.5f * PI) * Frj;
                    const float Gw = Fbar * PIw;
                    const float s1 = gk.x * dx + gk.y * dy + gk.z * dz;      // abar_k . d
                    const float s2 = -(gj.x * dx + gj.y * dy + gj.z * dz);   // abar_j . (x_k - x_j)
                    const float S = mj * s1 + mk * s2;
                    const float cw = S * Gw * rinv;
                    px += G * (mk * gj.x - mj * gk.x) - S * Gr * ux + cw * (vx + w * ux);
                    py += G * (mk * gj.y - mj * gk.y) - S * Gr * uy + cw * (vy + w * uy);
                    pz += G * (mk * gj.z - mj * gk.z) - S * Gr * uz + cw * (vz + w * uz);
                    ph += S * (Ak + 0.5f * PI) * Fhk;
                    pA += S * Fk;
                    pc += S * Fbar * PIc;
                    pr += S * Fbar * PIr;
                    pm += G * s2;
                } else if (PASS == 1) {
                    const float2 rdj = a.rd[q];
                    const float nj4 = kN * hinvj * hinvj * hinvj * hinvj;
                    // W_r = (8/pi) h^-4 w', W_hr = -(8/pi) h^-5 (4w' + q w''), W = (8/pi) h^-3 w,
                    // W_h = -(8/pi) h^-4 (3w + q w'), W_hh = (8/pi) h^-5 (12w + 8q w' + q^2 w'')
                    const float Wrk = nk4 * dwk, Wrj = nj4 * dwj;
                    const float Whrk = -nk4 * hinvk * (4.f * dwk + qk * ddwk);
                    const float Whrj = -nj4 * hinvj * (4.f * dwj + qj * ddwj);
                    const float coef = rdk.x * mj * Wrk + rdj.x * mk * Wrj + rdk.y * mj * Whrk + rdj.y * mk * Whrj;
                    px -= coef * ux;   // e_kj = -d-hat
                    py -= coef * uy;
                    pz -= coef * uz;
                    pm += rdj.x * (nj4 * hj * wj) + rdj.y * (-nj4 * (3.f * wj + qj * dwj));
                    ph += mj * nk4 * hinvk * (12.f * wk + 8.f * qk * dwk + qk * qk * ddwk);
                    pdN += qk * dwk;
                } else {
                    const float lj = a.lam[q];
                    const float coef = -(32.f / 3.f) * (lamk * dwk * hinvk + lj * dwj * hinvj);
                    px -= coef * ux;   // e_kj = -d-hat
                    py -= coef * uy;
                    pz -= coef * uz;
                }
            }
            kahan_add(Sx, Cx, px);
            kahan_add(Sy, Cy, py);
            kahan_add(Sz, Cz, pz);
            if (PASS <= 1) {
                kahan_add(Sm, Cm, pm);
                kahan_add(Sh, Ch, ph);
            }
            if (PASS == 0) {
                kahan_add(SA, CA, pA);
                kahan_add(Sc, Cc, pc);
                kahan_add(Sr, Cr, pr);
            }
            if (PASS == 1) kahan_add(SdN, CdN, pdN);
        }
        const float xs = Sx - Cx, ys = Sy - Cy, zs = Sz - Cz;
        if (PASS == 0) {
            const float Abar = SA - CA, cbar = Sc - Cc, hbarF = Sh - Ch;
            const float om = a.omega[k], uk = a.u[k];
            const float ubar = Abar * om * (gam - 1.f) / rhok + (ck > 0.f ? cbar * gam * (gam - 1.f) / (2.f * ck) : 0.f);
            const float Ombar = Abar * (gam - 1.f) * uk / rhok;
            const float D = 3.f * rhok * (1.f / om - 1.f) * hinvk;         // d rho / d h from Omega
            const float Bbar = -Ombar * om * om;
            const float rhobar = (Sr - Cr) - Abar * Ak / rhok + gk.w - Bbar * hk * D / (3.f * rhok * rhok);
            const float hbar = hbarF + Bbar * D / (3.f * rhok) + rhobar * D;
            a.xbar[k] = make_float4(xs, ys, zs, 0.f);
            a.mbar[k] = Sm - Cm;
            a.ubar[k] = ubar;
            a.hbar[k] = hbar;
            a.rd[k] = make_float2(rhobar, Bbar * hk / (3.f * rhok));
        } else if (PASS == 1) {
            // self terms of rho_k and D_k: W(0,h) = (8/pi) h^-3, W_h(0,h) = -3 (8/pi) h^-4,
            // W_hh(0,h) = 12 (8/pi) h^-5
            const float mbar = (Sm - Cm) + rdk.x * nk4 * hk - 3.f * rdk.y * nk4;
            const float hbar = a.hbar[k] + rdk.y * ((Sh - Ch) + 12.f * mk * nk4 * hinvk);
            const float dNdh = -(32.f / 3.f) * hinvk * (SdN - CdN);
            const float4 x0 = a.xbar[k];
            a.xbar[k] = make_float4(x0.x + xs, x0.y + ys, x0.z + zs, 0.f);
            a.mbar[k] += mbar;
            a.lam[k] = dNdh != 0.f ? hbar / dNdh : 0.f;
        } else {
            const float4 x0 = a.xbar[k];
            a.xbar[k] = make_float4(x0.x + xs, x0.y + ys, x0.z + zs, 0.f);
        }
    }
}

cudaError_t run_backward(sph_ctx* ctx, sph_grid* g, const BackwardLaunch& b, cudaStream_t s) {
    const int n = (int)g->n;
    if (!g->bw_ga) {
        cudaError_t e = cudaSuccess;
        if (!e) e = cudaMalloc(&g->bw_ga, sizeof(float4) * n);
        if (!e) e = cudaMalloc(&g->bw_xbar, sizeof(float4) * n);
        if (!e) e = cudaMalloc(&g->bw_rd, sizeof(float2) * n);
        if (!e) e = cudaMalloc(&g->bw_f, sizeof(float) * 6 * (size_t)n);
        if (e) return e;
    }
    grid_refresh_hmax(g, b.h, s);
    force_pack(g, b.vel, b.u, b.h, b.rho, b.omega, (float)b.gamma, s);
    ++ctx->launches;
    float* us = g->bw_f;
    float* oms = g->bw_f + n;
    float* mbar = g->bw_f + 2 * (size_t)n;
    float* ubar = g->bw_f + 3 * (size_t)n;
    float* hbar = g->bw_f + 4 * (size_t)n;
    float* lam = g->bw_f + 5 * (size_t)n;
    const int pb = (n + 255) / 256;
    k_bw_prep<<<pb, 256, 0, s>>>(n, g->perm, b.g_acc, b.g_rho, b.u, b.omega, g->bw_ga, us, oms);
    ++ctx->launches;
    BwArgs a;
    a.boxes = g->boxes;
    a.n_boxes = g->n_boxes;
    a.n = n;
    a.posm = g->posm;
    a.posf = g->posf;
    a.node_c = g->node_c;
    a.node_e = g->node_e;
    a.fvel = g->fvel;
    a.fthermo = g->fthermo;
    a.ga = g->bw_ga;
    a.u = us;
    a.omega = oms;
    a.xbar = g->bw_xbar;
    a.mbar = mbar;
    a.ubar = ubar;
    a.hbar = hbar;
    a.rd = g->bw_rd;
    a.lam = lam;
    a.alpha = (float)b.alpha;
    a.gamma = (float)b.gamma;
    const long long want = (n + kBwThreads - 1) / kBwThreads;
    const int blocks = (int)std::max<long long>(1, std::min<long long>(want, (long long)ctx->sm_count * 16));
    k_backward<0><<<blocks, kBwThreads, 0, s>>>(a);
    k_backward<1><<<blocks, kBwThreads, 0, s>>>(a);
    k_backward<2><<<blocks, kBwThreads, 0, s>>>(a);
    k_bw_scatter<<<pb, 256, 0, s>>>(n, g->perm, g->bw_xbar, ubar, mbar, b.g_pos, b.g_u, b.g_mass);
    ctx->launches += 4;
    return cudaGetLastError();
}

}  // namespace sph
