// abi.cu -- the extern "C" entry points declared in include/sph.h: argument
// validation on the host, dispatch to the kernels, and the device status word.
#include <cmath>
#include <cstring>

#include "internal.cuh"

using namespace sph;

namespace {

sph_status fail(sph_ctx* ctx, sph_status st, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return st;
}

sph_status cuda_fail(sph_ctx* ctx, cudaError_t e, const char* where) {
    return fail(ctx, e == cudaErrorMemoryAllocation ? SPH_ERR_OOM : SPH_ERR_CUDA,
                std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e));
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

sph_status check_params(sph_ctx* ctx, const sph_params* p) {
    if (!p) return fail(ctx, SPH_ERR_INVALID, "params is NULL");
    if (!finite_pos(p->box)) return fail(ctx, SPH_ERR_INVALID, "params.box must be finite and > 0");
    // N_eff(h) >= 32/3 (the particle's own w(0) term) for every h, so a
    // target at or below it has no root
    if (!finite_pos(p->n_target) || p->n_target <= 32.0 / 3.0)
        return fail(ctx, SPH_ERR_INVALID, "params.n_target must exceed 32/3 (the self term of N_eff)");
    if (!finite_pos(p->n_tol)) return fail(ctx, SPH_ERR_INVALID, "params.n_tol must be > 0");
    if (p->max_iter < 0 || p->max_iter > 10000) return fail(ctx, SPH_ERR_INVALID, "params.max_iter out of range");
    if (!std::isfinite(p->alpha_visc) || p->alpha_visc < 0) return fail(ctx, SPH_ERR_INVALID, "params.alpha_visc must be >= 0");
    if (!std::isfinite(p->gamma) || p->gamma <= 1.0) return fail(ctx, SPH_ERR_INVALID, "params.gamma must be > 1");
    if (p->group_size != 0 && (p->group_size < 8 || p->group_size > 4096 || (p->group_size & (p->group_size - 1))))
        return fail(ctx, SPH_ERR_INVALID, "params.group_size must be 0 (default) or a power of two in [8, 4096]");
    if (p->blocks_per_sm < 0 || p->blocks_per_sm > 32) return fail(ctx, SPH_ERR_INVALID, "params.blocks_per_sm out of range");
    if (!(p->walk_radius == 0.0 || (p->walk_radius >= 1.0 && p->walk_radius <= 2.0)))
        return fail(ctx, SPH_ERR_INVALID, "params.walk_radius must be 0 (default) or in [1, 2]");
    if ((p->flags & SPH_FP64) && (p->flags & SPH_PLAIN_FP32))
        return fail(ctx, SPH_ERR_INVALID, "SPH_FP64 and SPH_PLAIN_FP32 are exclusive");
    if (p->flags & (SPH_WARP_GROUP | SPH_COOP_WALK))
        return fail(ctx, SPH_ERR_INVALID, "SPH_WARP_GROUP and SPH_COOP_WALK name paths that are no longer built");
    if ((p->flags & SPH_WARP_WALK) &&
        (p->flags & (SPH_PER_THREAD_WALK | SPH_PLAIN_FP32 | SPH_FP64 | SPH_DENSITY_BUFFERED)))
        return fail(ctx, SPH_ERR_INVALID, "SPH_WARP_WALK excludes the other path flags and SPH_FP64");
    return SPH_OK;
}

// Which kernel family runs a density or force call. With no path flag the
// warp-per-particle kernels run (member-parallel for groups, one particle per
// warp for the rest): on the 10M clustered time bins they are the fastest at
// every active fraction measured (100, 10, 1 and 0.1 %). SPH_FP64 selects the
// per-thread walks in double.
enum class Path { Plain, Wpp, Thread };
Path pick_path(int flags) {
    if (flags & SPH_PLAIN_FP32) return Path::Plain;
    if (flags & (SPH_PER_THREAD_WALK | SPH_DENSITY_BUFFERED | SPH_FP64)) return Path::Thread;
    return Path::Wpp;
}

sph_status check_active(sph_ctx* ctx, const sph_grid* g, const int32_t* active, int64_t n_active) {
    if (active && (n_active < 0 || n_active > g->n))
        return fail(ctx, SPH_ERR_INVALID, "n_active must be in [0, n] when active is given");
    return SPH_OK;
}

}  // namespace

namespace sph {
cudaEvent_t timing_event(sph_ctx* ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
}  // namespace sph

extern "C" {

void sph_default_params(sph_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->box = 1.0;
    p->n_target = 64.0;
    p->n_tol = 64.0e-6;
    p->max_iter = 64;
    p->alpha_visc = 1.0;
    p->gamma = 5.0 / 3.0;
}

sph_status sph_create(sph_ctx** out, int device) {
    if (!out) return SPH_ERR_INVALID;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) return SPH_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return SPH_ERR_CUDA;
    sph_ctx* c = new sph_ctx();
    c->device = device;
    cudaError_t e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (!e) e = cudaMalloc(&c->counters, sizeof(Counters));
    if (!e) e = cudaMemset(c->counters, 0, sizeof(Counters));
    if (!e) e = cudaMalloc(&c->queue, sizeof(unsigned) * kQueues);
    if (!e) e = cudaMallocHost(&c->host_counters, sizeof(Counters));
    if (!e) e = cudaDeviceSynchronize();
    if (e) {
        sph_destroy(c);
        return e == cudaErrorMemoryAllocation ? SPH_ERR_OOM : SPH_ERR_CUDA;
    }
    *out = c;
    return SPH_OK;
}

void sph_destroy(sph_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->counters) cudaFree(c->counters);
    if (c->queue) cudaFree(c->queue);
    if (c->host_counters) cudaFreeHost(c->host_counters);
    for (auto& t : c->timed) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
    for (auto e : c->event_pool) cudaEventDestroy(e);
    delete c;
}

const char* sph_last_error(const sph_ctx* c) {
    if (!c) return "context is NULL";
    return c->err.c_str();
}

sph_status sph_build_grid_batched(sph_ctx* ctx, const void* pos, int pos_is_f64, const float* mass,
                                  const int64_t* box_offsets, const double* box_sizes, int n_boxes,
                                  const sph_params* params, void* stream, sph_grid** out) {
    if (!ctx) return SPH_ERR_INVALID;
    if (!out) return fail(ctx, SPH_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!pos || !mass) return fail(ctx, SPH_ERR_INVALID, "pos and mass must be device pointers");
    if (!box_offsets || !box_sizes || n_boxes < 1 || n_boxes > 65535)
        return fail(ctx, SPH_ERR_INVALID, "need 1..65535 boxes with host offsets and sizes");
    if (box_offsets[0] != 0) return fail(ctx, SPH_ERR_INVALID, "box_offsets[0] must be 0");
    for (int b = 0; b < n_boxes; ++b) {
        if (box_offsets[b + 1] <= box_offsets[b]) return fail(ctx, SPH_ERR_INVALID, "box_offsets must increase strictly");
        if (!finite_pos(box_sizes[b])) return fail(ctx, SPH_ERR_INVALID, "box sizes must be finite and > 0");
    }
    const int64_t n = box_offsets[n_boxes];
    if (n < 1 || n >= (int64_t(1) << 31)) return fail(ctx, SPH_ERR_INVALID, "total n must be in [1, 2^31)");
    sph_status st = check_params(ctx, params);
    if (st) return st;
    if (cudaSetDevice(ctx->device)) return fail(ctx, SPH_ERR_CUDA, "cudaSetDevice failed");
    return grid_build(ctx, pos, pos_is_f64 ? 1 : 0, mass, !(params->flags & SPH_NO_LISTS), box_offsets, box_sizes,
                      n_boxes, (cudaStream_t)stream, out);
}

sph_status sph_build_grid(sph_ctx* ctx, const void* pos, int pos_is_f64, const float* mass, int64_t n,
                          const sph_params* params, void* stream, sph_grid** out) {
    if (!ctx) return SPH_ERR_INVALID;
    sph_status st = check_params(ctx, params);
    if (st) return st;
    if (n < 1 || n >= (int64_t(1) << 31)) return fail(ctx, SPH_ERR_INVALID, "n must be in [1, 2^31)");
    int64_t offs[2] = {0, n};
    double L = params->box;
    return sph_build_grid_batched(ctx, pos, pos_is_f64, mass, offs, &L, 1, params, stream, out);
}

sph_status sph_grid_update(sph_ctx* ctx, sph_grid* grid, const void* pos, int pos_is_f64, const float* mass,
                           void* stream) {
    if (!ctx) return SPH_ERR_INVALID;
    if (!grid || grid->ctx != ctx) return fail(ctx, SPH_ERR_INVALID, "grid is NULL or from another context");
    if (!pos || !mass) return fail(ctx, SPH_ERR_INVALID, "pos and mass must be device pointers");
    if (cudaSetDevice(ctx->device)) return fail(ctx, SPH_ERR_CUDA, "cudaSetDevice failed");
    return grid_update(grid, pos, pos_is_f64 ? 1 : 0, mass, (cudaStream_t)stream);
}

void sph_grid_free(sph_grid* g) {
    if (!g) return;
    // the grid's own device: a grid may outlive its context (a garbage
    // collector finalises them in any order)
    cudaSetDevice(g->device);
    grid_free(g);
}

int64_t sph_grid_size(const sph_grid* g) { return g ? g->n : 0; }

sph_status sph_grid_export(const sph_grid* g, int32_t* perm, uint64_t* keys, uint32_t* X, void* stream) {
    if (!g) return SPH_ERR_INVALID;
    sph_ctx* ctx = g->ctx;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (perm && !e) e = cudaMemcpyAsync(perm, g->perm, sizeof(int32_t) * g->n, cudaMemcpyDeviceToDevice, s);
    if (keys && !e) e = cudaMemcpyAsync(keys, g->keys, sizeof(uint64_t) * g->n, cudaMemcpyDeviceToDevice, s);
    if (X && !e) e = cudaMemcpy2DAsync(X, 12, g->xq, 16, 12, g->n, cudaMemcpyDeviceToDevice, s);
    if (e) return cuda_fail(ctx, e, "sph_grid_export");
    return SPH_OK;
}

static sph_status density_call(sph_ctx* ctx, const sph_grid* grid, float* h, const int32_t* active,
                               int64_t n_active, float* rho, float* omega, int32_t* n_ngb, uint8_t* flags,
                               uint64_t* hash, const float* vel, float* divv, float* curlv,
                               const sph_params* params, void* stream) {
    if (!ctx) return SPH_ERR_INVALID;
    if (!grid || grid->ctx != ctx) return fail(ctx, SPH_ERR_INVALID, "grid is NULL or from another context");
    if (!h || !rho || !omega || !n_ngb || !flags) return fail(ctx, SPH_ERR_INVALID, "h, rho, omega, n_ngb, flags are required");
    sph_status st = check_params(ctx, params);
    if (st) return st;
    if ((st = check_active(ctx, grid, active, n_active))) return st;
    const int64_t na = active ? n_active : grid->n;
    if (na == 0) return SPH_OK;
    if (cudaSetDevice(ctx->device)) return fail(ctx, SPH_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)stream;
    sph_grid* g = const_cast<sph_grid*>(grid);  // per-call scratch lives in the grid
    const Path path = pick_path(params->flags);
    grid_active(g, active, n_active, s);
    DensityLaunch a;
    a.g = g;
    a.h = h;
    a.rho = rho;
    a.omega = omega;
    a.n_ngb = n_ngb;
    a.flags = flags;
    a.hash = reinterpret_cast<unsigned long long*>(hash);
    a.n_target = params->n_target;
    a.n_tol = params->n_tol;
    a.max_iter = params->max_iter;
    a.fixed_h = (params->flags & SPH_FIXED_H) ? 1 : 0;
    a.guess_h = (params->flags & SPH_H_GUESS) ? 1 : 0;
    a.fp64 = (params->flags & SPH_FP64) ? 1 : 0;
    a.blocks_per_sm = params->blocks_per_sm;
    a.walk_radius = params->walk_radius;
    a.group_span = params->group_size;
    a.time_kernels = (params->flags & SPH_TIME_KERNELS) ? 1 : 0;
    a.buffered = (params->flags & SPH_DENSITY_BUFFERED) ? 1 : 0;
    a.active_list = active ? 1 : 0;
    a.partial_lists = (params->flags & SPH_PARTIAL_LISTS) ? 1 : 0;
    a.vel = vel;
    a.divv = divv;
    a.curlv = curlv;
    g->lists_rec = false;   // set again by a call that records neighbour lists
    cudaError_t e = path == Path::Plain ? run_density_plain(ctx, a, na, s)
                    : path == Path::Wpp ? launch_density_wpp(ctx, a, na, s)
                                        : launch_density_tpp(ctx, a, na, s);
    if (!e) e = cudaGetLastError();
    if (e) return cuda_fail(ctx, e, "sph_density");
    return SPH_OK;
}

sph_status sph_density(sph_ctx* ctx, const sph_grid* grid, float* h, const int32_t* active, int64_t n_active,
                       float* rho, float* omega, int32_t* n_ngb, uint8_t* flags, uint64_t* hash,
                       const sph_params* params, void* stream) {
    return density_call(ctx, grid, h, active, n_active, rho, omega, n_ngb, flags, hash, nullptr, nullptr, nullptr,
                        params, stream);
}

sph_status sph_density_divcurl(sph_ctx* ctx, const sph_grid* grid, float* h, const int32_t* active,
                               int64_t n_active, float* rho, float* omega, int32_t* n_ngb, uint8_t* flags,
                               uint64_t* hash, const float* vel, float* divv, float* curlv,
                               const sph_params* params, void* stream) {
    if (!ctx) return SPH_ERR_INVALID;
    if (!vel || !divv || !curlv) return fail(ctx, SPH_ERR_INVALID, "vel, divv and curlv are required");
    if (params && pick_path(params->flags) != Path::Wpp)
        return fail(ctx, SPH_ERR_INVALID, "velocity divergence and curl run on the default path only");
    return density_call(ctx, grid, h, active, n_active, rho, omega, n_ngb, flags, hash, vel, divv, curlv, params,
                        stream);
}

static sph_status force_call(sph_ctx* ctx, const sph_grid* grid, const float* vel, const float* u,
                             const float* h, const float* rho, const float* omega, const float* divv,
                             const float* curlv, const float* kappa, const int32_t* active, int64_t n_active,
                             float* acc, float* dudt, float* vsig, float* dudt_cond, uint64_t* hash,
                             const sph_params* params, void* stream, const float* alpha_v = nullptr) {
    if (!ctx) return SPH_ERR_INVALID;
    if (!grid || grid->ctx != ctx) return fail(ctx, SPH_ERR_INVALID, "grid is NULL or from another context");
    if (!vel || !u || !h || !rho || !omega || !acc || !dudt || !vsig)
        return fail(ctx, SPH_ERR_INVALID, "vel, u, h, rho, omega, acc, dudt, vsig are required");
    sph_status st = check_params(ctx, params);
    if (st) return st;
    if ((st = check_active(ctx, grid, active, n_active))) return st;
    const int64_t na = active ? n_active : grid->n;
    if (na == 0) return SPH_OK;
    if (cudaSetDevice(ctx->device)) return fail(ctx, SPH_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)stream;
    sph_grid* g = const_cast<sph_grid*>(grid);
    const Path path = pick_path(params->flags & ~SPH_DENSITY_BUFFERED);
    grid_refresh_hmax(g, h, s);
    grid_active(g, active, n_active, s);
    ForceLaunch a;
    a.g = g;
    a.vel = vel;
    a.u = u;
    a.h = h;
    a.rho = rho;
    a.omega = omega;
    a.acc = acc;
    a.dudt = dudt;
    a.vsig = vsig;
    a.hash = reinterpret_cast<unsigned long long*>(hash);
    a.alpha = params->alpha_visc;
    a.gamma = params->gamma;
    a.fp64 = (params->flags & SPH_FP64) ? 1 : 0;
    a.blocks_per_sm = params->blocks_per_sm;
    a.group_span = params->group_size;
    a.time_kernels = (params->flags & SPH_TIME_KERNELS) ? 1 : 0;
    a.divv = divv;
    a.curlv = curlv;
    a.kappa = kappa;
    a.dudt_cond = dudt_cond;
    a.alpha_v = alpha_v;
    cudaError_t e = path == Path::Plain ? launch_force_plain(ctx, a, na, s)
                    : path == Path::Wpp ? launch_force_wpp(ctx, a, na, s)
                                        : launch_force_tpp(ctx, a, na, s);
    if (!e) e = cudaGetLastError();
    if (e) return cuda_fail(ctx, e, "sph_hydro_force");
    return SPH_OK;
}

sph_status sph_hydro_force(sph_ctx* ctx, const sph_grid* grid, const float* vel, const float* u,
                           const float* h, const float* rho, const float* omega, const int32_t* active,
                           int64_t n_active, float* acc, float* dudt, float* vsig, uint64_t* hash,
                           const sph_params* params, void* stream) {
    return force_call(ctx, grid, vel, u, h, rho, omega, nullptr, nullptr, nullptr, active, n_active, acc, dudt, vsig,
                      nullptr, hash, params, stream);
}

sph_status sph_hydro_force_balsara(sph_ctx* ctx, const sph_grid* grid, const float* vel, const float* u,
                                   const float* h, const float* rho, const float* omega, const float* divv,
                                   const float* curlv, const int32_t* active, int64_t n_active, float* acc,
                                   float* dudt, float* vsig, uint64_t* hash, const sph_params* params,
                                   void* stream) {
    if (!ctx) return SPH_ERR_INVALID;
    if (!divv || !curlv) return fail(ctx, SPH_ERR_INVALID, "divv and curlv are required");
    if (params && pick_path(params->flags & ~SPH_DENSITY_BUFFERED) != Path::Wpp)
        return fail(ctx, SPH_ERR_INVALID, "the Balsara switch runs on the default path only");
    return force_call(ctx, grid, vel, u, h, rho, omega, divv, curlv, nullptr, active, n_active, acc, dudt, vsig,
                      nullptr, hash, params, stream);
}

sph_status sph_hydro_force_visc(sph_ctx* ctx, const sph_grid* grid, const float* vel, const float* u, const float* h,
                                const float* rho, const float* omega, const float* alpha_v, const float* divv,
                                const float* curlv, const int32_t* active, int64_t n_active, float* acc, float* dudt,
                                float* vsig, uint64_t* hash, const sph_params* params, void* stream) {
    if (!ctx) return SPH_ERR_INVALID;
    if (!alpha_v) return fail(ctx, SPH_ERR_INVALID, "alpha_v is required");
    if ((divv == nullptr) != (curlv == nullptr)) return fail(ctx, SPH_ERR_INVALID, "give both divv and curlv, or neither");
    if (params && pick_path(params->flags & ~SPH_DENSITY_BUFFERED) != Path::Wpp)
        return fail(ctx, SPH_ERR_INVALID, "per-particle viscosity runs on the default path only");
    return force_call(ctx, grid, vel, u, h, rho, omega, divv, curlv, nullptr, active, n_active, acc, dudt, vsig,
                      nullptr, hash, params, stream, alpha_v);
}

sph_status sph_hydro_force_conduction(sph_ctx* ctx, const sph_grid* grid, const float* vel, const float* u,
                                      const float* h, const float* rho, const float* omega, const float* divv,
                                      const float* curlv, const float* kappa, const int32_t* active,
                                      int64_t n_active, float* acc, float* dudt, float* vsig, float* dudt_cond,
                                      uint64_t* hash, const sph_params* params, void* stream) {
    if (!ctx) return SPH_ERR_INVALID;
    if (!kappa || !dudt_cond) return fail(ctx, SPH_ERR_INVALID, "kappa and dudt_cond are required");
    if ((divv == nullptr) != (curlv == nullptr)) return fail(ctx, SPH_ERR_INVALID, "give both divv and curlv, or neither");
    if (params && pick_path(params->flags & ~SPH_DENSITY_BUFFERED) != Path::Wpp)
        return fail(ctx, SPH_ERR_INVALID, "conduction runs on the default path only");
    return force_call(ctx, grid, vel, u, h, rho, omega, divv, curlv, kappa, active, n_active, acc, dudt, vsig,
                      dudt_cond, hash, params, stream);
}

sph_status sph_gravity(sph_ctx* ctx, const sph_grid* grid, const int32_t* active, int64_t n_active,
                       const sph_gravity_params* gp, float* acc, int32_t* n_nodes, int32_t* n_pairs, void* stream) {
    if (!ctx) return SPH_ERR_INVALID;
    if (!grid || grid->ctx != ctx) return fail(ctx, SPH_ERR_INVALID, "grid is NULL or from another context");
    if (!gp || !acc) return fail(ctx, SPH_ERR_INVALID, "gp and acc are required");
    if (!(gp->theta >= 0.0 && gp->theta <= 1.0) || !(gp->r_split >= 0.0) || !(gp->h_soft >= 0.0) ||
        !std::isfinite(gp->G) || !std::isfinite(gp->r_split) || !std::isfinite(gp->h_soft) || !(gp->r_cut > 0.0))
        return fail(ctx, SPH_ERR_INVALID, "gravity: need 0 <= theta <= 1, r_split >= 0, h_soft >= 0, r_cut > 0");
    for (const auto& B : grid->boxes_h)
        if (!(gp->r_cut <= 0.25 * B.L)) return fail(ctx, SPH_ERR_INVALID, "gravity: r_cut must be <= L/4");
    sph_status st = check_active(ctx, grid, active, n_active);
    if (st) return st;
    const int64_t na = active ? n_active : grid->n;
    if (na == 0) return SPH_OK;
    if (cudaSetDevice(ctx->device)) return fail(ctx, SPH_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)stream;
    sph_grid* g = const_cast<sph_grid*>(grid);
    grid_active(g, active, n_active, s);
    GravityLaunch L;
    L.g = g;
    L.G = gp->G;
    L.theta = gp->theta;
    L.r_split = gp->r_split;
    L.r_cut = gp->r_cut;
    L.h_soft = gp->h_soft;
    L.acc = acc;
    L.n_nodes = n_nodes;
    L.n_pairs = n_pairs;
    cudaError_t e = launch_gravity(ctx, L, na, s);
    if (e) return cuda_fail(ctx, e, "sph_gravity");
    return SPH_OK;
}

sph_status sph_backward(sph_ctx* ctx, const sph_grid* grid, const float* vel, const float* u, const float* h,
                        const float* rho, const float* omega, const float* g_acc, const float* g_rho,
                        float* g_pos, float* g_u, float* g_mass, const sph_params* params, void* stream) {
    if (!ctx) return SPH_ERR_INVALID;
    if (!grid || grid->ctx != ctx) return fail(ctx, SPH_ERR_INVALID, "grid is NULL or from another context");
    if (!vel || !u || !h || !rho || !omega || !g_acc || !g_pos || !g_u || !g_mass)
        return fail(ctx, SPH_ERR_INVALID, "vel, u, h, rho, omega, g_acc, g_pos, g_u, g_mass are required");
    sph_status st = check_params(ctx, params);
    if (st) return st;
    if (params->flags & (SPH_FP64 | SPH_PLAIN_FP32 | SPH_WARP_GROUP))
        return fail(ctx, SPH_ERR_INVALID, "sph_backward runs the FP32 thread path only");
    if (cudaSetDevice(ctx->device)) return fail(ctx, SPH_ERR_CUDA, "cudaSetDevice failed");
    BackwardLaunch b;
    b.vel = vel;
    b.u = u;
    b.h = h;
    b.rho = rho;
    b.omega = omega;
    b.g_acc = g_acc;
    b.g_rho = g_rho;
    b.g_pos = g_pos;
    b.g_u = g_u;
    b.g_mass = g_mass;
    b.alpha = params->alpha_visc;
    b.gamma = params->gamma;
    cudaError_t e = run_backward(ctx, const_cast<sph_grid*>(grid), b, (cudaStream_t)stream);
    if (e) return cuda_fail(ctx, e, "sph_backward");
    return SPH_OK;
}

sph_status sph_sync_status(sph_ctx* ctx, void* stream, sph_stats* stats) {
    if (!ctx) return SPH_ERR_INVALID;
    if (cudaSetDevice(ctx->device)) return fail(ctx, SPH_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(ctx->host_counters, ctx->counters, sizeof(Counters), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemsetAsync(ctx->counters, 0, sizeof(Counters), s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return cuda_fail(ctx, e, "sph_sync_status");
    const Counters& c = *ctx->host_counters;
    double tms[2] = {0.0, 0.0};
    unsigned tn[2] = {0, 0};
    for (auto& t : ctx->timed) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
            tms[t.kind] += ms;
            tn[t.kind] += 1;
        }
        ctx->event_pool.push_back(t.a);
        ctx->event_pool.push_back(t.b);
    }
    ctx->timed.clear();
    const unsigned launches = ctx->launches;
    ctx->launches = 0;
    if (stats) {
        stats->status = c.status;
        stats->launches = launches;
        stats->density_kernel_ms = tms[0];
        stats->force_kernel_ms = tms[1];
        stats->density_launches = tn[0];
        stats->force_launches = tn[1];
        stats->density_pairs = c.density_pairs;
        stats->force_pairs = c.force_pairs;
        stats->density_evals = c.density_evals;
        stats->pair_tests = c.pair_tests;
        stats->groups = c.groups;
        stats->list_force = c.list_force;
        stats->grav_nodes = c.grav_nodes;
        stats->grav_pairs = c.grav_pairs;
    }
    if (c.status & ST_INVALID) return fail(ctx, SPH_ERR_INVALID, "device: non-finite or out-of-range input");
    if (c.status & ST_TIMEOUT) return fail(ctx, SPH_ERR_TIMEOUT, "device: a bounded wait ran out");
    if (c.status & ST_H_TOO_LARGE) return fail(ctx, SPH_ERR_H_TOO_LARGE, "device: some h reached L/2");
    if (c.status & ST_NOT_CONVERGED) return fail(ctx, SPH_ERR_NOT_CONVERGED, "device: some h did not converge");
    return SPH_OK;
}

}  // extern "C"
