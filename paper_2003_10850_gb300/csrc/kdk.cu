// kdk.cu -- kick-drift-kick time integration with power-of-two time bins.
//
// The paper's code advances particles on individual, power-of-two time steps
// (Sec. 2.2): at each step only the particles whose step ends are active,
// and the others (inactive neighbours included) are drifted to the current
// time. These kernels are the device side of that bookkeeping:
//   k_timebins      bin of each particle from its Courant step dt = C h / v_sig
//   k_active_flags  which particles end a step at integer time `tick`
//   k_kick          v += a dt_bin, u += du/dt dt_bin for the active particles
//                   (optionally copying the kicked values to the predictions)
//   k_drift         x += v dt for every particle (FP64 positions, periodic), and
//                   the predictions v_pred += a dt, u_pred += du/dt dt that the
//                   next force evaluations use
//   k_visc_rate     d alpha/dt of the time-dependent viscosity (Morris & Monaghan)
//   k_kick_scalar,  the same kick and prediction for one more per-particle
//   k_predict_scalar  quantity (the viscosity parameter)
// The integer timeline counts steps of the smallest bin, dt_max / 2^max_bin;
// a particle in bin b has step dt_max / 2^b and ends a step at every tick that
// is a multiple of 2^(max_bin - b).
#include <cmath>

#include "internal.cuh"

namespace sph {

// Bin of a Courant step: the smallest b in [0, max_bin] with dt_max <= dt 2^b
// (exact comparisons: scaling by 2^b is exact in FP32), max_bin if none; then
// raised until the new step starts on a boundary of its bin at `tick`.
__global__ void k_timebins(int n, const float* __restrict__ h, const float* __restrict__ vsig,
                           const int32_t* __restrict__ active, int na, float courant, float dt_max, int max_bin,
                           long long tick, uint8_t* __restrict__ bins) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (active ? na : n)) return;
    const int i = active ? active[t] : t;
    if (i < 0 || i >= n) return;   // padding entry of a fixed-capacity list
    const float vs = vsig[i];
    int b = 0;
    if (vs > 0.f) {
        const float dt = __fdiv_rn(__fmul_rn(courant, h[i]), vs);
        while (b < max_bin && !(dt_max <= ldexpf(dt, b))) ++b;
    }
    while (b < max_bin && (tick & ((1ll << (max_bin - b)) - 1)) != 0) ++b;
    bins[i] = (uint8_t)b;
}

__global__ void k_active_flags(int n, const uint8_t* __restrict__ bins, long long tick, int max_bin,
                               uint8_t* __restrict__ flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = min((int)bins[i], max_bin);
    flag[i] = (tick & ((1ll << (max_bin - b)) - 1)) == 0 ? 1 : 0;
}

// The active particles ascending in active[0, count), then -1 in every entry
// of active[count, n): the whole array can be passed on with n_active = n,
// without reading the count on the host (negative entries are skipped).
__global__ void k_flags_to_list(int n, const uint8_t* __restrict__ flag, const uint32_t* __restrict__ scan,
                                int32_t* __restrict__ active, int32_t* __restrict__ count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        if (flag[i]) active[scan[i]] = i;
        else active[scan[n] + (i - scan[i])] = -1;
    }
    if (i == 0) *count = (int32_t)scan[n];
}

struct KickSteps {
    float dt[32];
};

__global__ void k_kick(int na, const int32_t* __restrict__ active, const uint8_t* __restrict__ bins, KickSteps ks,
                       int n_bins, const float* __restrict__ acc, const float* __restrict__ dudt,
                       float* __restrict__ vel, float* __restrict__ u, float* __restrict__ vel_pred,
                       float* __restrict__ u_pred) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= na) return;
    const int i = active[t];
    if (i < 0) return;   // padding entry of a fixed-capacity list
    const float dt = ks.dt[min((int)bins[i], n_bins - 1)];
    const size_t k = 3 * (size_t)i;
    const float vx = fmaf(acc[k], dt, vel[k]), vy = fmaf(acc[k + 1], dt, vel[k + 1]),
                vz = fmaf(acc[k + 2], dt, vel[k + 2]), uu = fmaf(dudt[i], dt, u[i]);
    vel[k] = vx;
    vel[k + 1] = vy;
    vel[k + 2] = vz;
    u[i] = uu;
    if (vel_pred) {
        vel_pred[k] = vx;
        vel_pred[k + 1] = vy;
        vel_pred[k + 2] = vz;
        u_pred[i] = uu;
    }
}

// x += v dt in FP64, wrapped into [0, L); v_pred += a dt, u_pred += du/dt dt.
// invL > 0: L is a power of two and invL = 1/L exactly, so x * invL is x / L
// without the FP64 division.
__global__ void k_drift(int n, double* __restrict__ pos, const float* __restrict__ vel, double dt, double L,
                        double invL, const float* __restrict__ acc, const float* __restrict__ dudt,
                        float* __restrict__ vel_pred, float* __restrict__ u_pred) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * n) return;
    double x = fma((double)vel[t], dt, pos[t]);
    x -= L * floor(invL > 0.0 ? x * invL : x / L);
    if (x >= L) x -= L;
    pos[t] = x;
    if (vel_pred) {
        const float dtf = (float)dt;
        vel_pred[t] = fmaf(acc[t], dtf, vel_pred[t]);
        if (t < n) u_pred[t] = fmaf(dudt[t], dtf, u_pred[t]);
    }
}

// d alpha/dt = -(alpha - alpha_min) ell c / h + max(-div v, 0) (alpha_max - alpha),
// c = sqrt(gamma (gamma - 1) u): decay to alpha_min over tau = h / (ell c),
// growth towards alpha_max where the flow converges (Morris & Monaghan 1997).
__global__ void k_visc_rate(int na, const int32_t* __restrict__ active, const float* __restrict__ h,
                            const float* __restrict__ u, const float* __restrict__ divv,
                            const float* __restrict__ alpha, float gg1, float amin, float amax, float ell,
                            float* __restrict__ dalpha) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= na) return;
    const int i = active ? active[t] : t;
    if (i < 0) return;   // padding entry of a fixed-capacity list
    const float c = sqrtf(gg1 * u[i]);
    const float a = alpha[i];
    dalpha[i] = fmaxf(-divv[i], 0.f) * (amax - a) - (a - amin) * (ell * c / h[i]);
}

__global__ void k_kick_scalar(int na, const int32_t* __restrict__ active, const uint8_t* __restrict__ bins,
                              KickSteps ks, int n_bins, const float* __restrict__ rate, float* __restrict__ value,
                              float* __restrict__ value_pred) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= na) return;
    const int i = active[t];
    if (i < 0) return;   // padding entry of a fixed-capacity list
    const float v = fmaf(rate[i], ks.dt[min((int)bins[i], n_bins - 1)], value[i]);
    value[i] = v;
    if (value_pred) value_pred[i] = v;
}

__global__ void k_predict_scalar(int n, float dt, const float* __restrict__ rate, float* __restrict__ value_pred) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) value_pred[i] = fmaf(rate[i], dt, value_pred[i]);
}

}  // namespace sph

using namespace sph;

namespace {
sph_status kdk_fail(sph_ctx* ctx, sph_status st, const char* msg) {
    if (ctx) ctx->err = msg;
    return st;
}
}  // namespace

sph_status sph_timebins(sph_ctx* ctx, const float* h, const float* vsig, const int32_t* active, int64_t n_active,
                        int64_t n, int64_t tick, double courant, double dt_max, int max_bin, uint8_t* bins,
                        void* stream) {
    if (!ctx) return SPH_ERR_INVALID;
    if (!h || !vsig || !bins || n < 1 || n >= (int64_t(1) << 31) || (active && (n_active < 0 || n_active > n)))
        return kdk_fail(ctx, SPH_ERR_INVALID, "sph_timebins: bad pointers or sizes");
    if (!(courant > 0.0) || !(dt_max > 0.0) || max_bin < 0 || max_bin > 30 || tick < 0)
        return kdk_fail(ctx, SPH_ERR_INVALID, "sph_timebins: courant, dt_max > 0, 0 <= max_bin <= 30, tick >= 0");
    if (cudaSetDevice(ctx->device)) return kdk_fail(ctx, SPH_ERR_CUDA, "cudaSetDevice failed");
    const int cnt = (int)(active ? n_active : n);
    if (cnt == 0) return SPH_OK;
    cudaStream_t s = (cudaStream_t)stream;
    k_timebins<<<(cnt + 255) / 256, 256, 0, s>>>((int)n, h, vsig, active, cnt, (float)courant, (float)dt_max,
                                                 max_bin, (long long)tick, bins);
    ++ctx->launches;
    return cudaGetLastError() ? kdk_fail(ctx, SPH_ERR_CUDA, "sph_timebins launch failed") : SPH_OK;
}

sph_status sph_active_from_bins(sph_ctx* ctx, sph_grid* grid, const uint8_t* bins, int64_t tick, int max_bin,
                                int32_t* active, int32_t* n_active, void* stream) {
    if (!ctx) return SPH_ERR_INVALID;
    if (!grid || grid->ctx != ctx || !bins || !active || !n_active)
        return kdk_fail(ctx, SPH_ERR_INVALID, "sph_active_from_bins: bad grid or pointers");
    if (max_bin < 0 || max_bin > 30 || tick < 0)
        return kdk_fail(ctx, SPH_ERR_INVALID, "sph_active_from_bins: 0 <= max_bin <= 30, tick >= 0");
    if (cudaSetDevice(ctx->device)) return kdk_fail(ctx, SPH_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = (int)grid->n;
    k_active_flags<<<(n + 255) / 256, 256, 0, s>>>(n, bins, (long long)tick, max_bin, grid->flag);
    scan_exclusive<uint8_t>(grid->flag, n, grid->scan, grid->scan_tmp, s, &ctx->launches);
    k_flags_to_list<<<(n + 255) / 256, 256, 0, s>>>(n, grid->flag, grid->scan, active, n_active);
    ctx->launches += 2;
    return cudaGetLastError() ? kdk_fail(ctx, SPH_ERR_CUDA, "sph_active_from_bins launch failed") : SPH_OK;
}

sph_status sph_kick(sph_ctx* ctx, const int32_t* active, int64_t n_active, const uint8_t* bins, const double* dt_bin,
                    int n_bins, const float* acc, const float* dudt, float* vel, float* u, float* vel_pred,
                    float* u_pred, void* stream) {
    if (!ctx) return SPH_ERR_INVALID;
    if (!active || !bins || !dt_bin || !acc || !dudt || !vel || !u || n_bins < 1 || n_bins > 32 || n_active < 0 ||
        n_active >= (int64_t(1) << 31) || (vel_pred == nullptr) != (u_pred == nullptr))
        return kdk_fail(ctx, SPH_ERR_INVALID, "sph_kick: bad pointers or sizes (1 <= n_bins <= 32)");
    if (cudaSetDevice(ctx->device)) return kdk_fail(ctx, SPH_ERR_CUDA, "cudaSetDevice failed");
    if (n_active == 0) return SPH_OK;
    KickSteps ks = {};
    for (int b = 0; b < n_bins; ++b) ks.dt[b] = (float)dt_bin[b];
    cudaStream_t s = (cudaStream_t)stream;
    k_kick<<<(int)((n_active + 255) / 256), 256, 0, s>>>((int)n_active, active, bins, ks, n_bins, acc, dudt, vel, u,
                                                         vel_pred, u_pred);
    ++ctx->launches;
    return cudaGetLastError() ? kdk_fail(ctx, SPH_ERR_CUDA, "sph_kick launch failed") : SPH_OK;
}

sph_status sph_drift(sph_ctx* ctx, double* pos, const float* vel, int64_t n, double dt, double box,
                     const float* acc, const float* dudt, float* vel_pred, float* u_pred, void* stream) {
    if (!ctx) return SPH_ERR_INVALID;
    if (!pos || !vel || n < 1 || n >= (int64_t(1) << 30) || !(box > 0.0) || !std::isfinite(dt))
        return kdk_fail(ctx, SPH_ERR_INVALID, "sph_drift: bad pointers, n, box or dt");
    const bool pred = vel_pred || u_pred || acc || dudt;
    if (pred && !(vel_pred && u_pred && acc && dudt))
        return kdk_fail(ctx, SPH_ERR_INVALID, "sph_drift: give acc, dudt, vel_pred and u_pred together, or none");
    if (cudaSetDevice(ctx->device)) return kdk_fail(ctx, SPH_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)stream;
    const int m = (int)(3 * n);
    int ex = 0;
    const double invL = std::frexp(box, &ex) == 0.5 ? 1.0 / box : 0.0;
    k_drift<<<(m + 255) / 256, 256, 0, s>>>((int)n, pos, vel, dt, box, invL, acc, dudt, vel_pred, u_pred);
    ++ctx->launches;
    return cudaGetLastError() ? kdk_fail(ctx, SPH_ERR_CUDA, "sph_drift launch failed") : SPH_OK;
}

sph_status sph_visc_rate(sph_ctx* ctx, const int32_t* active, int64_t n_active, const float* h, const float* u,
                         const float* divv, const float* alpha_v, double gamma, double alpha_min, double alpha_max,
                         double ell, float* dalpha, void* stream) {
    if (!ctx) return SPH_ERR_INVALID;
    if (!h || !u || !divv || !alpha_v || !dalpha || n_active < 0 || n_active >= (int64_t(1) << 31))
        return kdk_fail(ctx, SPH_ERR_INVALID, "sph_visc_rate: bad pointers or n_active");
    if (!(gamma > 1.0) || !(ell > 0.0) || !(alpha_min >= 0.0) || !(alpha_max >= alpha_min))
        return kdk_fail(ctx, SPH_ERR_INVALID, "sph_visc_rate: gamma > 1, ell > 0, 0 <= alpha_min <= alpha_max");
    if (cudaSetDevice(ctx->device)) return kdk_fail(ctx, SPH_ERR_CUDA, "cudaSetDevice failed");
    if (n_active == 0) return SPH_OK;
    cudaStream_t s = (cudaStream_t)stream;
    k_visc_rate<<<(int)((n_active + 255) / 256), 256, 0, s>>>((int)n_active, active, h, u, divv, alpha_v,
                                                              (float)(gamma * (gamma - 1.0)), (float)alpha_min,
                                                              (float)alpha_max, (float)ell, dalpha);
    ++ctx->launches;
    return cudaGetLastError() ? kdk_fail(ctx, SPH_ERR_CUDA, "sph_visc_rate launch failed") : SPH_OK;
}

sph_status sph_kick_scalar(sph_ctx* ctx, const int32_t* active, int64_t n_active, const uint8_t* bins,
                           const double* dt_bin, int n_bins, const float* rate, float* value, float* value_pred,
                           void* stream) {
    if (!ctx) return SPH_ERR_INVALID;
    if (!active || !bins || !dt_bin || !rate || !value || n_bins < 1 || n_bins > 32 || n_active < 0 ||
        n_active >= (int64_t(1) << 31))
        return kdk_fail(ctx, SPH_ERR_INVALID, "sph_kick_scalar: bad pointers or sizes (1 <= n_bins <= 32)");
    if (cudaSetDevice(ctx->device)) return kdk_fail(ctx, SPH_ERR_CUDA, "cudaSetDevice failed");
    if (n_active == 0) return SPH_OK;
    KickSteps ks = {};
    for (int b = 0; b < n_bins; ++b) ks.dt[b] = (float)dt_bin[b];
    cudaStream_t s = (cudaStream_t)stream;
    k_kick_scalar<<<(int)((n_active + 255) / 256), 256, 0, s>>>((int)n_active, active, bins, ks, n_bins, rate, value,
                                                                value_pred);
    ++ctx->launches;
    return cudaGetLastError() ? kdk_fail(ctx, SPH_ERR_CUDA, "sph_kick_scalar launch failed") : SPH_OK;
}

sph_status sph_predict_scalar(sph_ctx* ctx, int64_t n, double dt, const float* rate, float* value_pred,
                              void* stream) {
    if (!ctx) return SPH_ERR_INVALID;
    if (!rate || !value_pred || n < 1 || n >= (int64_t(1) << 31) || !std::isfinite(dt))
        return kdk_fail(ctx, SPH_ERR_INVALID, "sph_predict_scalar: bad pointers, n or dt");
    if (cudaSetDevice(ctx->device)) return kdk_fail(ctx, SPH_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)stream;
    k_predict_scalar<<<(int)((n + 255) / 256), 256, 0, s>>>((int)n, (float)dt, rate, value_pred);
    ++ctx->launches;
    return cudaGetLastError() ? kdk_fail(ctx, SPH_ERR_CUDA, "sph_predict_scalar launch failed") : SPH_OK;
}
