// internal.cuh -- host-side structures shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "common.cuh"
#include "sph.h"

struct sph_ctx {
    int device = 0;
    int sm_count = 0;
    std::string err;
    sph::Counters* counters = nullptr;  // device
    unsigned* queue = nullptr;          // device work-queue counters (kQueues)
    sph::Counters* host_counters = nullptr;  // pinned
    unsigned launches = 0;                   // kernels launched since the last sync
    // SPH_TIME_KERNELS: event pairs around the main kernels (kind 0 density, 1 force)
    struct Timed { cudaEvent_t a, b; int kind; };
    std::vector<Timed> timed;
    std::vector<cudaEvent_t> event_pool;
};

struct sph_grid {
    sph_ctx* ctx = nullptr;
    int device = 0;                        // the context's device: freeing needs no live context
    int64_t n = 0;
    int n_boxes = 0;
    int box_bits = 0;
    int n_nodes = 0;
    int max_leaves = 0;                    // max over boxes of level-0 nodes
    int max_lev = 0;                       // max over boxes of the level count
    int lvl_max[sph::kMaxLev] = {};        // max over boxes of the nodes on each level
    std::vector<sph::BoxDesc> boxes_h;
    sph::BoxDesc* boxes = nullptr;         // device
    uint4* posm = nullptr;                 // sorted: X, Y, Z, mass bits
    uint4* xq = nullptr;                   // caller order: X, Y, Z, mass bits
    int32_t* perm = nullptr;               // sorted -> caller
    int32_t* rank = nullptr;               // caller -> sorted
    uint64_t* keys = nullptr;              // sorted keys
    uint4* node_lo = nullptr;
    uint4* node_hi = nullptr;
    float* node_hmax = nullptr;
    uint4* node_c = nullptr;               // node centre (integer)
    float4* node_e = nullptr;              // node half extents (box units), w = h_max
    float4* posf = nullptr;                // sorted: leaf-relative position (box units), mass
    float4* fvel = nullptr;                // per force call, sorted: v, h
    float4* fthermo = nullptr;             // per force call, sorted: rho, A, c, 1/h
    float4* fposh = nullptr;               // per force call, sorted: leaf-relative position, h
    float4* fvm = nullptr;                 // per force call, sorted: v, m
    float* fbal = nullptr;                 // per force call with the switch, sorted: Balsara factor
    float2* fcond = nullptr;               // per force call with conduction, sorted: u, kappa
    float2* fvisc = nullptr;               // per force call with per-particle viscosity, sorted: factor, alpha
    float4* node_m = nullptr;              // per gravity call, per node: centre of mass - node centre, mass
    unsigned long long* box_rci = nullptr; // per gravity call, per box: coarse squared cutoff
    // per-call scratch, sized at build so that calls never allocate
    int32_t* act = nullptr;                // active particles, sorted indices, sorted order
    uint8_t* flag = nullptr;               // n
    uint32_t* scan = nullptr;              // n + 1
    uint32_t* scan_tmp = nullptr;          // block sums
    // plain-path scratch
    int32_t* list_a = nullptr;
    int32_t* list_b = nullptr;
    float* st_lo = nullptr;
    float* st_hi = nullptr;
    int* list_n = nullptr;                 // device [2]
    // rebuild scratch (kept so that sph_grid_update never allocates)
    long long* d_off = nullptr;
    double* d_L = nullptr;
    unsigned long long* k2 = nullptr;
    unsigned* v1 = nullptr;
    unsigned* v2 = nullptr;
    unsigned* counts = nullptr;
    unsigned* cscan = nullptr;
    int32_t* mp_j = nullptr;               // density, member-parallel path: near-list indices per persistent warp
    int32_t* den_left = nullptr;           // density: particles left to the one-particle kernel (n)
    // neighbour lists recorded by an all-active density call on the default path and
    // reused by the force pass (NULL when the grid was built with SPH_NO_LISTS)
    int32_t* nbr = nullptr;                // pool of kListPool * n entries: the lists {j != i : r_ij < h_i}
    int32_t* nbr_off = nullptr;            // n: start of i's list in the pool
    int32_t* nbr_n = nullptr;              // n: length of i's list, -1 if the pool was full
    uint32_t* ext_n = nullptr;             // n: extra partners of i (j with h_i <= r_ij < h_j); after
                                           // the sort, kExtUnusable if they overflowed their segment
    int32_t* ext = nullptr;                // n segments of kExtCap: i's extra partners, ascending
    uint4* list_xh = nullptr;              // n: integer position and the bits of the h the lists were
                                           // made with (sorted order): one gather for the transpose
    unsigned* list_st = nullptr;           // device, kListSt words (see kListSt)
    int32_t* fb_list = nullptr;            // n: active particles the list force pass hands to the walk
    bool lists_rec = false;                // host: the last density call recorded lists (all or some particles)
    uint32_t* list_ep = nullptr;           // n: generation (list_st word kListGen) of the call that recorded
                                           // the particle's list and extra partners
    int32_t* mp_x = nullptr;               // density, member-parallel path of a partial call: per warp,
                                           // kMpMembers x kMpFar inactive partners beyond the near radius
    int64_t list_pool = 0;                 // entries of the nbr pool
    // adjoint scratch (allocated by the first sph_backward on the grid)
    float4* bw_ga = nullptr;
    float4* bw_xbar = nullptr;
    float2* bw_rd = nullptr;
    float* bw_f = nullptr;
};

namespace sph {

constexpr int kQueues = 8;
constexpr int kListPool = 128;  // neighbour-list pool entries per particle (lists vary in length)
constexpr int kExtCap = 128;    // extra-partner segment per particle (262k clustered: mean 24, max 106)
constexpr unsigned kExtUnusable = 0xffffffffu;
static_assert((kExtCap & (kExtCap - 1)) == 0 && kExtCap >= 64, "kExtCap: a power of two >= 64 (the segment sort)");
constexpr int kListChunk = 2048; // pool entries a warp reserves at a time for its particles' lists
// density, member-parallel path: members per group (the largest work chunk),
// near-list entries per member, resident warps per SM at most
constexpr int kMpMembers = 8;
constexpr int kMpCap = 128;
constexpr int kMpWarpsPerSm = 64;
// list_st words: [0] lists written, [1] a list missing (pool full) or the
// extra partners incomplete, [2] h changed since the lists were made, [3]
// fallback count, [4..5] pool entries reserved (64-bit), [6] generation: one
// more for every density call (never cleared), [7] unused
constexpr int kListSt = 8;
constexpr int kListGen = 6;
constexpr int kMpFar = 128;     // inactive partners beyond the near radius per member (partial calls)

// grid.cu
sph_status grid_build(sph_ctx* ctx, const void* pos, int f64, const float* mass, bool lists,
                      const int64_t* offs, const double* Ls, int nb, cudaStream_t s,
                      sph_grid** out);
void grid_free(sph_grid* g);
// re-quantise, re-sort and rebuild the hierarchy in place (same n and boxes)
sph_status grid_update(sph_grid* g, const void* pos, int f64, const float* mass, cudaStream_t s);
// hmax of every node from the caller-order h
void grid_refresh_hmax(sph_grid* g, const float* h, cudaStream_t s);
// active list: sorted indices in g->act, count in g->scan[n]
void grid_active(sph_grid* g, const int32_t* active, int64_t n_active, cudaStream_t s);
// exclusive scan of n values into out[0..n] (out[n] = total); tmp >= n/4096+2 words
template <typename In>
void scan_exclusive(const In* in, int n, uint32_t* out, uint32_t* tmp, cudaStream_t s, unsigned* launches);
// SPH_TIME_KERNELS support: event pair around one kernel launch
cudaEvent_t timing_event(sph_ctx* ctx);

// the density pass (launch descriptions shared by the paths)
struct DensityLaunch {
    const sph_grid* g;
    float* h;
    float* rho;
    float* omega;
    int32_t* n_ngb;
    uint8_t* flags;
    unsigned long long* hash;
    double n_target, n_tol;
    int max_iter;
    int fixed_h, guess_h;
    int fp64;
    int blocks_per_sm;
    double walk_radius;   // 0: default
    int group_span = 0;   // sorted particles a group stays within (power of two; 0: default)
    int time_kernels;
    int buffered;
    int active_list = 0;  // the caller gave an active list (the device count may be below n_active)
    int partial_lists = 0; // SPH_PARTIAL_LISTS
    // velocity divergence and curl at the final h (default path only; NULL: not asked)
    const float* vel = nullptr;
    float* divv = nullptr;
    float* curlv = nullptr;
};
// plain.cu
cudaError_t run_density_plain(sph_ctx* ctx, const DensityLaunch& a, int64_t n_active,
                              cudaStream_t s);

// the force pass
struct ForceLaunch {
    const sph_grid* g;
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
    int fp64;
    int blocks_per_sm;
    int group_span = 0;   // as DensityLaunch
    int time_kernels;
    // Balsara's switch (default path only; NULL: no switch)
    const float* divv = nullptr;
    const float* curlv = nullptr;
    // thermal conduction (default path only; NULL: none): conductivity in, heating rate out
    const float* kappa = nullptr;
    float* dudt_cond = nullptr;
    // per-particle viscosity parameter (default path only; NULL: alpha for every pair)
    const float* alpha_v = nullptr;
};
cudaError_t launch_force_plain(sph_ctx* ctx, const ForceLaunch& a, int64_t n_active,
                               cudaStream_t s);

// backward.cu
struct BackwardLaunch {
    const float* vel;
    const float* u;
    const float* h;
    const float* rho;
    const float* omega;
    const float* g_acc;
    const float* g_rho;
    float* g_pos;
    float* g_u;
    float* g_mass;
    double alpha, gamma;
};
cudaError_t run_backward(sph_ctx* ctx, sph_grid* g, const BackwardLaunch& b, cudaStream_t s);


// gravity.cu
struct GravityLaunch {
    const sph_grid* g;
    double G, theta, r_split, r_cut, h_soft;
    float* acc;
    int32_t* n_nodes;   // optional
    int32_t* n_pairs;   // optional
};
cudaError_t launch_gravity(sph_ctx* ctx, const GravityLaunch& L, int64_t n_active, cudaStream_t s);

// wpp_density.cu, wpp_force.cu (one warp per particle)
cudaError_t launch_density_wpp(sph_ctx* ctx, const DensityLaunch& a, int64_t n_active, cudaStream_t s);
cudaError_t launch_force_wpp(sph_ctx* ctx, const ForceLaunch& a, int64_t n_active, cudaStream_t s);

// tpp.cu (per-thread walks)
// list_xh / h_changed (optional): set *h_changed if some h differs from the h in list_xh;
// divv / curlv (optional, caller order): Balsara factors into g->fbal;
// kappa (optional, caller order): (u, kappa) into g->fcond;
// alpha_v (optional, caller order): (Balsara factor or 1, alpha) into g->fvisc
void force_pack(const sph_grid* g, const float* vel, const float* u, const float* h, const float* rho,
                const float* omega, float gamma, cudaStream_t s, const uint4* list_xh = nullptr,
                unsigned* h_changed = nullptr, const float* divv = nullptr, const float* curlv = nullptr,
                const float* kappa = nullptr, const float* alpha_v = nullptr);
cudaError_t launch_density_tpp(sph_ctx* ctx, const DensityLaunch& a, int64_t n_active, cudaStream_t s);
cudaError_t launch_force_tpp(sph_ctx* ctx, const ForceLaunch& a, int64_t n_active, cudaStream_t s);

}  // namespace sph
