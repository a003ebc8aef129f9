/*
 * sph.h -- C ABI of the GB300 SPH neighbour-interaction library
 * (libsph_gb300.so). Plain pointers and sizes only: no CUDA, PyTorch or C++
 * types cross this boundary. `stream` arguments are cudaStream_t values passed
 * as void* (NULL = the legacy default stream).
 *
 * The library implements the data-parallel hot path of the SPH part of
 * "Gadget3 on GPUs with OpenACC" (Ragagnin et al. 2020): the two SPH modules
 * -- an iterated density pass and a hydrodynamic-force pass (Sec. 1) -- over
 * the neighbours within a fixed distance of each active particle (Sec. 1,
 * Sec. 2.4), for the uneven active sets that adaptive time bins produce
 * (Sec. 2.2). The paper states no SPH formula; the library follows the
 * standard Gadget-2 forms, spelled out at each entry point.
 *
 * Ownership: every particle array is a caller-owned DEVICE pointer indexed in
 * the caller's particle order, except where marked "host". The library owns
 * sph_ctx and sph_grid and every workspace they hold. Outputs are written only
 * for active particles; other entries are left untouched.
 *
 * Errors: every call validates its arguments on the host and returns a
 * status synchronously; kernels run asynchronously on `stream`. Conditions
 * found on the device (non-convergence, h >= L/2, non-finite input, a bounded
 * wait that ran out) set bits in a device status word that sph_sync_status()
 * returns. Nothing here traps or aborts; no exception crosses the ABI.
 * sph_last_error() holds a message for the last non-OK status.
 */
#ifndef SPH_GB300_H
#define SPH_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPH_OK = 0,
    SPH_ERR_INVALID = 1,        /* bad argument (host check) or non-finite input (device) */
    SPH_ERR_CUDA = 2,           /* a CUDA runtime call failed; see sph_last_error() */
    SPH_ERR_NOT_CONVERGED = 3,  /* some h did not converge within max_iter (device) */
    SPH_ERR_H_TOO_LARGE = 4,    /* some h would reach L/2 (minimum image breaks) (device) */
    SPH_ERR_TIMEOUT = 5,        /* a bounded device-side wait ran out (device) */
    SPH_ERR_OOM = 6             /* device allocation failed */
} sph_status;

/* sph_params.flags */
#define SPH_FP64       0x01  /* pair arithmetic and sums in FP64 (the plain method in double) */
#define SPH_PLAIN_FP32 0x02  /* plain path: thread per particle, FP32, no compensation,
                                h iterated by the host (the baseline the fast path is measured against) */
#define SPH_FIXED_H    0x04  /* density: evaluate at the given h, do not iterate */
#define SPH_H_GUESS    0x08  /* density: ignore the h input and start from a local
                                estimate made from the grid's leaf-parent boxes */
#define SPH_TIME_KERNELS 0x10 /* record CUDA events around the main density/force kernel on
                                 the launching stream; sph_sync_status sums their durations */
#define SPH_WARP_GROUP 0x20   /* reserved: names a path that is no longer built (SPH_ERR_INVALID) */
#define SPH_DENSITY_BUFFERED 0x40 /* density, per-thread walks: iterate h on a per-thread buffer
                                     of the candidates found by one walk at 1.06 h */
#define SPH_PER_THREAD_WALK 0x80  /* force one thread per particle walking alone */
#define SPH_WARP_WALK 0x200       /* one warp per active particle (the default path when no other
                                     path flag is given): the warp walks for its particle (four
                                     nodes per step, one child per lane), keeps the leaf list in
                                     shared memory across h iterations, tests 32 candidates per step
                                     and evaluates the pair terms from a warp-wide hit buffer */
#define SPH_COOP_WALK 0x100       /* reserved: names a path that is no longer built (SPH_ERR_INVALID) */
#define SPH_NO_LISTS 0x400        /* sph_build_grid: do not allocate the neighbour lists that the
                                     default path records in an all-active density pass and reuses
                                     in the force pass (saves ~1,040 bytes per particle) */
#define SPH_PARTIAL_LISTS 0x800   /* sph_density on the default path with an active list of at least
                                     n/256 entries (the member-parallel kernel then runs whatever the
                                     count): record the active particles' lists
                                     and their extra partners (j with h_i <= r_ij < h_j), those
                                     among the inactive particles found by a wider sweep of the
                                     density pass, so that a force call on that set reads them.
                                     The wider sweep costs the density pass about what the lists
                                     save the force pass; without the flag such a call records
                                     nothing and the force pass walks. */

/* Device status bits returned in sph_stats.status */
#define SPH_ST_NOT_CONVERGED 0x01
#define SPH_ST_H_TOO_LARGE   0x02
#define SPH_ST_TIMEOUT       0x04
#define SPH_ST_INVALID       0x08

typedef struct sph_ctx sph_ctx;    /* opaque, library-owned */
typedef struct sph_grid sph_grid;  /* opaque, library-owned */

typedef struct {
    double box;         /* periodic box side L (sph_build_grid); > 0 */
    double n_target;    /* N_t: target of N_eff(h) = (4 pi/3) h^3 sum_j W(r_ij,h), self included */
    double n_tol;       /* converged when |N_eff - N_t| <= n_tol */
    int    max_iter;    /* h iterations per particle before SPH_ST_NOT_CONVERGED */
    double alpha_visc;  /* artificial-viscosity alpha */
    double gamma;       /* adiabatic index */
    int    flags;       /* SPH_* flags above */
    int    group_size;  /* default path: a group of the member-parallel kernels (up to 8 active
                           particles sharing one walk) never leaves an aligned run of this many
                           sorted particles: 0 = library default (64, a leaf-parent node), else a
                           power of two in [8, 4096]. Larger spans make fuller groups of sparse
                           active sets with larger boxes. */
    int    blocks_per_sm; /* persistent CTAs per SM: 0 = library default */
    double walk_radius; /* density, default path: radius of a particle's candidate (near) list
                           as a multiple of its starting h, in [1, 2]; 0 = library default
                           (1.04). Larger radii keep more candidates but walk again less
                           often when h grows during the iteration. */
} sph_params;

/* Counters accumulated by the device since the last sph_sync_status(). */
typedef struct {
    uint32_t status;          /* OR of SPH_ST_* bits */
    uint32_t launches;        /* kernels launched by this context (host count) */
    uint64_t density_pairs;   /* sum over active i of n_ngb,i at the converged h */
    uint64_t force_pairs;     /* sum over active i of |{j != i : r_ij < max(h_i, h_j)}| */
    uint64_t density_evals;   /* particle-evaluations of the density sums (all iterations) */
    uint64_t pair_tests;      /* candidate pairs tested (work including rejected ones) */
    uint64_t groups;          /* reserved (0) */
    double density_kernel_ms; /* SPH_TIME_KERNELS: summed time of the density kernels */
    double force_kernel_ms;   /* SPH_TIME_KERNELS: summed time of the force kernels */
    uint32_t density_launches; /* SPH_TIME_KERNELS: timed density kernel launches */
    uint32_t force_launches;   /* SPH_TIME_KERNELS: timed force kernel launches */
    uint64_t grav_nodes;      /* sph_gravity: node (monopole) interactions */
    uint64_t grav_pairs;      /* sph_gravity: particle interactions inside the cutoff */
    uint64_t list_force;      /* force: active particles served from the neighbour lists that
                                 the last density call recorded (the others walk) */
} sph_stats;

/* Fills *p with the library defaults: L = 1, N_t = 64, n_tol = 1e-6 N_t,
 * max_iter = 64, alpha = 1, gamma = 5/3, flags = 0. */
void sph_default_params(sph_params *p);

/* Creates a context on CUDA device `device` (made current). */
sph_status sph_create(sph_ctx **ctx, int device);
void sph_destroy(sph_ctx *ctx);
/* Message for the last non-OK status of calls on ctx (never NULL). */
const char *sph_last_error(const sph_ctx *ctx);

/*
 * Quantise, key, sort and build the neighbour grid of one periodic box
 * (paper Sec. 1: each module walks a tree built over the particles; here the
 * tree is a Morton-ordered bounding-volume hierarchy built on the GPU).
 *   pos   device, n x 3 (x,y,z interleaved), float (pos_is_f64 = 0) or double
 *         (pos_is_f64 = 1); any finite value, wrapped into [0, L).
 *         Quantisation: X = rint(frac(x/L) 2^32) mod 2^32 per axis (round half
 *         to even); all geometry after this point is exact integer geometry,
 *         minimum image d = (int32)(X_j - X_i).
 *   mass  device, n floats (> 0); copied into the grid (sorted order), so
 *         the caller may free or change it afterwards.
 *   n     1 <= n < 2^31.
 * Keys: 63-bit Morton key of the top 21 bits per axis (x most significant in
 * each triple); sort: stable by (key, caller index). On success *out is a new
 * grid (free with sph_grid_free). Non-finite positions set SPH_ST_INVALID.
 */
sph_status sph_build_grid(sph_ctx *ctx, const void *pos, int pos_is_f64, const float *mass,
                          int64_t n, const sph_params *params, void *stream, sph_grid **out);

/*
 * As sph_build_grid for many independent periodic boxes in one grid (and so
 * in one launch per pass). Box b holds the caller particles
 * [box_offsets[b], box_offsets[b+1]) and has side box_sizes[b].
 *   box_offsets  HOST, n_boxes + 1 int64, box_offsets[0] = 0, strictly
 *                increasing, box_offsets[n_boxes] = total n.
 *   box_sizes    HOST, n_boxes doubles > 0.
 * Keys carry the box index in their top ceil(log2 n_boxes) bits and the
 * Morton key shifted down by as many bits below it.
 */
sph_status sph_build_grid_batched(sph_ctx *ctx, const void *pos, int pos_is_f64,
                                  const float *mass, const int64_t *box_offsets,
                                  const double *box_sizes, int n_boxes,
                                  const sph_params *params, void *stream, sph_grid **out);

/*
 * Rebuild an existing grid in place for new positions/masses of the same
 * particles (same n and box layout): quantise, key, sort and bound again,
 * asynchronously on `stream`, with no allocation and no host synchronisation
 * -- the per-step rebuild of a time-stepping loop, capturable in a CUDA graph.
 * Argument meaning as in sph_build_grid.
 */
sph_status sph_grid_update(sph_ctx *ctx, sph_grid *grid, const void *pos, int pos_is_f64,
                           const float *mass, void *stream);

/* Frees a grid (NULL: nothing). Needs no live context: a grid may be freed
 * after the context that built it was destroyed. */
void sph_grid_free(sph_grid *grid);
int64_t sph_grid_size(const sph_grid *grid);

/*
 * Test/inspection access to the grid (device outputs, any may be NULL):
 *   perm  n int32: caller index of the k-th particle in sorted order;
 *   keys  n uint64: sorted keys;
 *   X     n x 3 uint32: quantised positions in CALLER order.
 */
sph_status sph_grid_export(const sph_grid *grid, int32_t *perm, uint64_t *keys, uint32_t *X,
                           void *stream);

/*
 * Density pass with on-device smoothing-length iteration (paper Sec. 1: the
 * first of the two SPH modules, which iterates until each h settles).
 * For each active i (the caller indices in `active[0..n_active)`, device
 * int32; a repeated index counts once and negative entries are skipped, so a
 * list padded with -1 up to a fixed capacity -- as sph_active_from_bins
 * writes it -- can be passed whole without reading its count on the host;
 * active = NULL means all particles):
 *   h_i solves N_eff(h) = (4 pi/3) h^3 sum_j W(r_ij, h) = N_t (self included,
 *   W = M4 cubic spline with support h) to |N_eff - N_t| <= n_tol (or until
 *   the bracket is one float wide: h is stored in FP32), by a bracketed,
 *   bisection-safeguarded Newton iteration on N_eff^(1/3), starting from h[i]
 *   (in/out, box units);
 *   rho_i   = sum_j m_j W(r_ij, h_i)                (self included)
 *   omega_i = [1 + h_i/(3 rho_i) d rho_i/d h_i]^-1  (grad-h factor)
 *   n_ngb_i = #{j != i : r_ij < h_i} under the exact predicate
 *             (double)D2 < (h 2^32/L)^2, D2 the exact integer squared distance.
 *   flags_i = SPH_ST_NOT_CONVERGED / SPH_ST_H_TOO_LARGE bits for i (uint8).
 *   hash_i  = optional (NULL to skip) checksum of the neighbour set:
 *             sum over j of splitmix64(caller index j), mod 2^64.
 * With SPH_FIXED_H the sums are evaluated once at the given h.
 * Arithmetic (default path): FP32 pair terms; per-lane FP32 partial sums
 * folded across the lanes that share a particle by error-free (TwoSum)
 * transformations and rounded once; the h update in FP32 on the compensated
 * N_eff; FP64 only in the exact neighbour predicate, for the rare pairs
 * within 2^-20 of the radius. SPH_PER_THREAD_WALK keeps an FP64 bracket and
 * h update; SPH_FP64 computes everything in FP64.
 * Neighbour lists (default path, grid built without SPH_NO_LISTS): when every
 * particle is active the call records each particle's set {j != i : r_ij <
 * h_i} at its final h in the grid, and, for each i, the partners j with
 * h_i <= r_ij < h_j (the transpose), so that a following sph_hydro_force can
 * take its pairs from these lists (see there). A call on a smaller active set
 * records nothing (the force pass then walks), unless SPH_PARTIAL_LISTS is
 * given: then each active particle's list and extra partners are recorded
 * and stamped with the call, and the lists of the particles that were not
 * active in it stop serving the force pass.
 */
sph_status sph_density(sph_ctx *ctx, const sph_grid *grid, float *h, const int32_t *active,
                       int64_t n_active, float *rho, float *omega, int32_t *n_ngb,
                       uint8_t *flags, uint64_t *hash, const sph_params *params, void *stream);

/*
 * Hydrodynamic-force pass (paper Sec. 1, the second SPH module), grad-h
 * Gadget-2 form in specific internal energy u. Inputs are indexed by caller
 * order for ALL particles (neighbours may be inactive):
 *   vel (n x 3), u, h, rho, omega (n each) device floats.
 * For each active i, over j != i with r_ij < max(h_i, h_j):
 *   P = (gamma-1) rho u,  c = sqrt(gamma P/rho),  A = omega P / rho^2,
 *   w_ij = v_ij . r_ij / r,  v_sig = c_i + c_j - 3 w_ij,
 *   Pi_ij = -(alpha/2) v_sig w_ij / ((rho_i+rho_j)/2) if w_ij < 0 else 0,
 *   acc_i  = -sum_j m_j [A_i gradW_ij(h_i) + A_j gradW_ij(h_j) + Pi_ij gradbarW_ij]
 *   dudt_i =  A_i sum_j m_j v_ij.gradW_ij(h_i) + 1/2 sum_j m_j Pi_ij v_ij.gradbarW_ij
 *   vsig_i = max(0, max_j v_sig);  coincident pairs (r = 0) add no force.
 * acc is n x 3. hash (optional) is the pair-set checksum as in sph_density.
 * Sums are folded error-free across the lanes that share a particle and
 * rounded once.
 * Pair source (default path): if the last sph_density call on this grid
 * recorded lists (every particle active, or SPH_PARTIAL_LISTS), the grid has
 * not been updated since, and every h equals the h that call ended with
 * (checked on the device), the pairs of each active particle whose list that
 * call recorded come from the lists -- no hierarchy walk, no candidate test.
 * The other active particles (not active in that call, or whose lists did not
 * fit: the neighbour pool full, or more than 128 extra partners) walk the
 * hierarchy, and so does the whole active set when the lists cannot serve the
 * call. Both give the same pair set.
 */
sph_status sph_hydro_force(sph_ctx *ctx, const sph_grid *grid, const float *vel, const float *u,
                           const float *h, const float *rho, const float *omega,
                           const int32_t *active, int64_t n_active, float *acc, float *dudt,
                           float *vsig, uint64_t *hash, const sph_params *params, void *stream);

/*
 * Velocity divergence and curl for Balsara's viscosity switch (the paper's
 * code runs an "improved SPH", Sec. 1; the forms are Gadget-2's, which
 * estimates them in its density loop). The density pass of sph_density
 * (default path only: no path flag), plus, for each active i, over its
 * neighbour set {j != i : r_ij < h_i} at the final h:
 *   divv_i  = -(1/rho_i) sum_j m_j v_ij . grad_i W_ij(h_i)
 *   curlv_i = |(1/rho_i) sum_j m_j v_ij x grad_i W_ij(h_i)|
 * with v_ij = v_i - v_j, r_ij = x_i - x_j, grad_i W_ij = dW/dr r_ij/r_ij.
 *   vel    device, n x 3 floats (caller order, all particles);
 *   divv, curlv  device, n floats: written for active particles.
 * Other arguments, outputs and the neighbour-list recording as sph_density.
 * SPH_ERR_INVALID for a missing pointer or a path flag.
 */
sph_status sph_density_divcurl(sph_ctx *ctx, const sph_grid *grid, float *h, const int32_t *active,
                               int64_t n_active, float *rho, float *omega, int32_t *n_ngb, uint8_t *flags,
                               uint64_t *hash, const float *vel, float *divv, float *curlv,
                               const sph_params *params, void *stream);

/*
 * sph_hydro_force with Balsara's switch on the artificial viscosity
 * (default path only):
 *   f_i = |divv_i| / (|divv_i| + curlv_i + 1e-4 c_i/h_i),
 *   Pi_ij -> Pi_ij (f_i + f_j)/2,
 * so the viscosity fades where the flow is shear-dominated. divv and curlv
 * are device arrays of n floats for all particles (caller order), e.g. from
 * sph_density_divcurl. Everything else as sph_hydro_force (same pair source:
 * the recorded neighbour lists when they match).
 */
sph_status sph_hydro_force_balsara(sph_ctx *ctx, const sph_grid *grid, const float *vel, const float *u,
                                   const float *h, const float *rho, const float *omega, const float *divv,
                                   const float *curlv, const int32_t *active, int64_t n_active, float *acc,
                                   float *dudt, float *vsig, uint64_t *hash, const sph_params *params,
                                   void *stream);

/*
 * sph_hydro_force with a viscosity parameter per particle (time-dependent
 * artificial viscosity, the "improved SPH" viscosity of the paper's code,
 * Sec. 1; default path only): the pair takes alpha_ij = (alpha_i + alpha_j)/2
 * in place of params->alpha_visc,
 *   Pi_ij = -(alpha_ij/2) v_sig w_ij / rho_bar [(f_i + f_j)/2],
 * the bracket (Balsara's switch) when divv and curlv are given.
 *   alpha_v      device, n floats (caller order, all particles);
 *   divv, curlv  both NULL (no switch) or as in sph_hydro_force_balsara.
 * Everything else as sph_hydro_force. alpha_v usually evolves with
 * sph_visc_rate, sph_kick_scalar and sph_predict_scalar.
 */
sph_status sph_hydro_force_visc(sph_ctx *ctx, const sph_grid *grid, const float *vel, const float *u, const float *h,
                                const float *rho, const float *omega, const float *alpha_v, const float *divv,
                                const float *curlv, const int32_t *active, int64_t n_active, float *acc, float *dudt,
                                float *vsig, uint64_t *hash, const sph_params *params, void *stream);

/*
 * The force pass plus thermal conduction over the same pair set, in one
 * traversal (default path only). The paper's code has a conduction module
 * that loops over neighbours like the force module (Sec. 1); the paper
 * states no formula, so this is the SPH conduction of Cleary & Monaghan
 * (1999), as Jubelgas, Springel & Dolag (2004) used it in Gadget, for u with a
 * conductivity kappa per particle (heat flux -kappa grad u):
 *   dudt_cond_i = sum_j m_j/(rho_i rho_j) 4 kappa_i kappa_j/(kappa_i + kappa_j)
 *                 (u_i - u_j) Fbar_ij,
 *   Fbar_ij = (F(r_ij, h_i) + F(r_ij, h_j))/2,  F(r, h) = dW/dr(r, h)/r,
 * over j != i with r_ij < max(h_i, h_j). The pair terms are antisymmetric, so
 * sum_i m_i dudt_cond_i = 0 over an all-active pass.
 *   kappa      device, n floats (>= 0, caller order, all particles);
 *   dudt_cond  device, n floats: written for active particles (separate from
 *              dudt, which stays the hydrodynamic rate);
 *   divv, curlv  both NULL (no switch) or as in sph_hydro_force_balsara.
 * Everything else as sph_hydro_force.
 */
sph_status sph_hydro_force_conduction(sph_ctx *ctx, const sph_grid *grid, const float *vel, const float *u,
                                      const float *h, const float *rho, const float *omega, const float *divv,
                                      const float *curlv, const float *kappa, const int32_t *active,
                                      int64_t n_active, float *acc, float *dudt, float *vsig, float *dudt_cond,
                                      uint64_t *hash, const sph_params *params, void *stream);

/*
 * Time integration on individual power-of-two time steps (the paper's
 * adaptive time bins, Sec. 2.2): kick-drift-kick with the bookkeeping on the
 * device. The integer timeline counts steps of the smallest bin,
 * dt_max / 2^max_bin ("ticks"); a particle in bin b has step dt_max / 2^b and
 * ends a step at every tick that is a multiple of 2^(max_bin - b).
 *
 * sph_timebins: bins from the Courant step dt_i = courant * h_i / vsig_i (FP32,
 * correctly rounded): the smallest b in [0, max_bin] with dt_max <= dt_i 2^b
 * (max_bin if none; 0 if vsig_i <= 0), then raised until tick is a multiple of
 * 2^(max_bin - b) (a new step starts on its bin's boundary). For the active
 * particles (caller indices, device) or all (active = NULL). h, vsig device
 * floats, bins device uint8 (n each, caller order).
 */
sph_status sph_timebins(sph_ctx *ctx, const float *h, const float *vsig, const int32_t *active, int64_t n_active,
                        int64_t n, int64_t tick, double courant, double dt_max, int max_bin, uint8_t *bins,
                        void *stream);
/* The particles that end a step at `tick`, ascending (caller indices) into
 * active[0, count) (device, capacity n), then -1 in every later entry up to n;
 * the count into *n_active (device int32). The padded list can be passed
 * whole (n_active = n) to the density, force and kick calls, which skip
 * negative entries: a time-stepping loop then never reads the count on the
 * host and can be captured in a CUDA graph. Uses the grid's scratch (the
 * grid fixes n). */
sph_status sph_active_from_bins(sph_ctx *ctx, sph_grid *grid, const uint8_t *bins, int64_t tick, int max_bin,
                                int32_t *active, int32_t *n_active, void *stream);
/* Kick: for each active i (negative entries of active skipped),
 * v_i += a_i dt_bin[bins_i] and u_i += dudt_i dt_bin[bins_i]
 * (FP32 fused multiply-add). dt_bin is a HOST array of n_bins (<= 32) steps.
 * vel_pred, u_pred (both or neither): also receive the kicked values (after a
 * closing half kick these are the synchronized velocity and energy, the
 * starting point of the next predictions). */
sph_status sph_kick(sph_ctx *ctx, const int32_t *active, int64_t n_active, const uint8_t *bins,
                    const double *dt_bin, int n_bins, const float *acc, const float *dudt, float *vel, float *u,
                    float *vel_pred, float *u_pred, void *stream);
/* Drift: x += v dt for all n particles, in FP64, wrapped into [0, box). pos is
 * device n x 3 doubles, vel device n x 3 floats. With acc, dudt, vel_pred,
 * u_pred (all four or none): also v_pred += a dt and u_pred += dudt dt, the
 * predictions at the new time that the force evaluations take (the force
 * depends on v through the viscosity and on u through the pressure). */
sph_status sph_drift(sph_ctx *ctx, double *pos, const float *vel, int64_t n, double dt, double box,
                     const float *acc, const float *dudt, float *vel_pred, float *u_pred, void *stream);

/* Rate of the per-particle viscosity parameter (Morris & Monaghan 1997), for
 * the active particles (caller indices, device) or all (active = NULL):
 *   dalpha_i = -(alpha_i - alpha_min) ell c_i / h_i + max(-divv_i, 0) (alpha_max - alpha_i),
 *   c_i = sqrt(gamma (gamma - 1) u_i),
 * a decay to alpha_min over tau = h/(ell c) (h the support radius) and a
 * source where the flow converges. h, u, divv, alpha_v, dalpha: device, n
 * floats, caller order. SPH_ERR_INVALID unless gamma > 1, ell > 0 and
 * 0 <= alpha_min <= alpha_max. */
sph_status sph_visc_rate(sph_ctx *ctx, const int32_t *active, int64_t n_active, const float *h, const float *u,
                         const float *divv, const float *alpha_v, double gamma, double alpha_min, double alpha_max,
                         double ell, float *dalpha, void *stream);
/* sph_kick for one per-particle quantity: value_i += rate_i dt_bin[bins_i]
 * for the active particles; value_pred (or NULL) also receives the result. */
sph_status sph_kick_scalar(sph_ctx *ctx, const int32_t *active, int64_t n_active, const uint8_t *bins,
                           const double *dt_bin, int n_bins, const float *rate, float *value, float *value_pred,
                           void *stream);
/* The prediction of sph_drift for one quantity: value_pred += rate dt, all n. */
sph_status sph_predict_scalar(sph_ctx *ctx, int64_t n, double dt, const float *rate, float *value_pred,
                              void *stream);

/*
 * Short-range gravity of the TreePM split by a Barnes-Hut walk (the paper's
 * gravity module: particles interact with distant tree nodes as point masses
 * chosen by an opening criterion, inside the walk; Sec. 1, Sec. 3). The long-
 * range particle-mesh part is not computed here.
 *   tree      the grid's hierarchy: a leaf is 8 consecutive Morton-sorted
 *             particles, a node 8 consecutive nodes of the level below; node
 *             boxes are the min/max integer coordinates of their particles,
 *             node masses and centres of mass the sums (computed by the call).
 *   decisions exact integer comparisons in coarse units (integer
 *             coordinates >> 8): with D2 the squared periodic gap between X_i
 *             and a node's box, F2 the squared distance to its far side
 *             (rounded up), L2 its squared largest side, RCi =
 *             ceil((r_cut 2^24 / L)^2) and P = rint(theta^2 2^16), the root is
 *             opened and a child of an opened node is skipped if D2 >= RCi,
 *             taken as its monopole if P > 0, D2 > 0, F2 < RCi, L2 <= D2 and
 *             2^16 L2 <= P D2, else opened; a particle j != i of an opened leaf
 *             interacts if sum_a (|(int32)(X_j - X_i)| >> 8)^2 < RCi.
 *   term      a_i += G m_j K(r) (x_j - x_i) (minimum image; a node: its mass at
 *             its centre of mass), K(r) = M(r/h_soft) g(r) / r^3 with M the mass
 *             fraction of the cubic spline (support h_soft) inside r (1 beyond,
 *             or with h_soft = 0) and g(r) = erfc(r/(2 r_split)) +
 *             r/(r_split sqrt(pi)) exp(-r^2/(4 r_split^2)) (1 with r_split = 0).
 *             Coincident pairs exert nothing.
 *   active    device int32 caller indices (NULL: all), as sph_density;
 *   acc       device, n x 3 floats: written for active particles (FP32 sums
 *             folded with error-free transformations);
 *   n_nodes, n_pairs  device, n int32 each, or NULL: per active particle the
 *             node and particle interactions.
 * SPH_ERR_INVALID unless 0 <= theta <= 1, r_split >= 0, h_soft >= 0, G
 * finite and 0 < r_cut <= L/4 for every box of the grid. The totals are in
 * sph_stats.grav_nodes / grav_pairs.
 */
typedef struct {
    double G;        /* gravitational constant */
    double theta;    /* opening angle (0: never accept a node) */
    double r_split;  /* TreePM split scale r_s (0: no split) */
    double r_cut;    /* cutoff radius, <= L/4 */
    double h_soft;   /* spline softening radius (support; 0: none) */
} sph_gravity_params;
sph_status sph_gravity(sph_ctx *ctx, const sph_grid *grid, const int32_t *active, int64_t n_active,
                       const sph_gravity_params *gp, float *acc, int32_t *n_nodes, int32_t *n_pairs, void *stream);

/*
 * Adjoint of the density and force passes (an extension of the paper's hot
 * path, which has no gradients). All particles are active. Given the forward
 * state of the grid's particles -- vel, u (inputs of the force pass) and h,
 * rho, omega as sph_density returned them with h converged (N_eff(h) = N_t) --
 * and the seeds
 *   g_acc  device, n x 3: dL/da_i;   g_rho  device, n, or NULL (zero): dL/drho_i,
 * writes dL/dx (g_pos, n x 3), dL/du (g_u, n) and dL/dm (g_mass, n) through
 * the whole chain: the implicit dependence of h on the positions
 * (dh/dx = -(dN/dx)/(dN/dh)), rho and d rho/dh, the grad-h factor Omega, the
 * pressure and viscosity terms. Velocities are constants. The pair sets are
 * recomputed by walking the grid (no neighbour lists are stored). FP32 pair
 * terms with compensated sums; deterministic (gathers, no atomics). The
 * first call on a grid allocates its adjoint workspace (~56 bytes/particle).
 */
sph_status sph_backward(sph_ctx *ctx, const sph_grid *grid, const float *vel, const float *u,
                        const float *h, const float *rho, const float *omega, const float *g_acc,
                        const float *g_rho, float *g_pos, float *g_u, float *g_mass,
                        const sph_params *params, void *stream);

/*
 * Stable sort of 64-bit keys that allocates nothing (the paper has no
 * counterpart: this serves callers that cannot call cudaMalloc -- code that
 * runs inside another framework's memory pool or budget, time-critical loops
 * where cudaMalloc's implicit synchronisation is not acceptable, or callers
 * without a sph_ctx, whose creation allocates).
 *   keys         device, n uint64 (read only);
 *   sorted_keys  device, n uint64: the keys in ascending order;
 *   perm         device, n int32: perm[k] = index of the k-th smallest key,
 *                equal keys in index order (stable) -- the same order
 *                sph_build_grid sorts its Morton keys in;
 *   1 <= n <= SPH_SORT_STATIC_MAX_KEYS, else SPH_ERR_INVALID (also for NULL
 *   pointers); SPH_ERR_CUDA if a CUDA call fails.
 * Runs asynchronously on `stream` on the current device. Its scratch is a
 * fixed device array of about 12.6 MB inside the library, which every GPU
 * that uses it holds until the process exits. Every call looks up that
 * array's address in the current context (no allocation), so a context that
 * was reset and created again is handled. Set-up: under lazy module loading
 * (CUDA_MODULE_LOADING=LAZY, CUDA's default) the array is created when this
 * module is first used on a device -- by the first call, unless another
 * kernel of the library ran there before -- which allocates and may
 * synchronise; make that first call before any stream capture and outside
 * any memory budget. All calls on a device share the array: calls whose
 * kernels overlap on the GPU (different streams, or different host threads)
 * race and corrupt each other's results -- serialise them. Nothing needs
 * clearing between calls: every scratch word a call reads it wrote itself.
 * SPH_ERR_CUDA, without launching, if a CUDA error is already pending on the
 * calling thread (it is left pending for its owner).
 */
#define SPH_SORT_STATIC_MAX_KEYS (1 << 20)
sph_status sph_sort_keys_static(const uint64_t *keys, int64_t n, uint64_t *sorted_keys,
                                int32_t *perm, void *stream);

/*
 * Waits for `stream`, then returns the device status word and counters
 * accumulated since the previous call in *stats (may be NULL) and clears
 * them. Returns the sph_status of the worst device condition seen.
 */
sph_status sph_sync_status(sph_ctx *ctx, void *stream, sph_stats *stats);

#ifdef __cplusplus
}
#endif

#endif /* SPH_GB300_H */
