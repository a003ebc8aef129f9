/*
 * sph_oracle.c -- plain FP64 CPU oracle for the SPH density and hydro-force
 * passes and the short-range gravity pass. TEST INFRASTRUCTURE ONLY: it is loaded by tests/, by the
 * __graft_entry__ smoke check and by the CPU-baseline leg of bench.py, and by
 * nothing else. It shares no code, header or constant with the CUDA library.
 *
 * What it computes (the paper names the two SPH modules -- an iterated density
 * pass and a force pass -- and that neighbours lie within a fixed distance,
 * Sec. 1 and Sec. 2.4, but states no formula; the formulas below are the
 * standard Gadget-2-style SPH the paper's code descends from):
 *
 *   positions   X = rint(frac(x/L) * 2^32) mod 2^32 per axis (uint32), minimum
 *               image d = (int32)(X_j - X_i) (two's-complement wrap).
 *   kernel      M4 cubic spline with support h:
 *                 W(r,h) = 8/(pi h^3) w(q), q = r/h,
 *                 w = 1 - 6q^2 + 6q^3 (q <= 1/2), 2(1-q)^3 (1/2 < q < 1), 0 else.
 *   predicate   j is a neighbour of i at h  <=>  (double)D2 < H*H, with
 *               D2 = dx^2+dy^2+dz^2 exact in uint64 (integer units) and
 *               H = h * 2^32 / L in FP64.
 *   h           root of N_eff(h) = (4 pi/3) h^3 sum_j W(r_ij,h) = N_t (self
 *               included), found by bracketed Newton/bisection.
 *   density     rho_i = sum_j m_j W(r_ij,h_i); drho/dh = sum_j m_j dW/dh;
 *               Omega_i = 1 / (1 + h_i/(3 rho_i) drho/dh);
 *               n_ngb = #{j != i : neighbour}.
 *   force       P = (gamma-1) rho u, c = sqrt(gamma P / rho), A = Omega P / rho^2,
 *               pair set j != i with r < max(h_i, h_j),
 *               w_ij = v_ij . r_ij / |r_ij|, v_sig = c_i + c_j - 3 w_ij,
 *               Pi_ij = -(alpha/2) v_sig w_ij / rho_bar if w_ij < 0 else 0,
 *               a_i   = -sum_j m_j [A_i grad W(h_i) + A_j grad W(h_j) + Pi_ij gradbar W],
 *               du_i  =  A_i sum_j m_j v_ij . grad W(h_i)
 *                        + 1/2 sum_j m_j Pi_ij v_ij . gradbar W,
 *               vsig_i = max(0, max_j v_sig).
 *   switch      (optional) velocity divergence and curl from the density
 *               pass's neighbours, div_i = -(1/rho_i) sum_j m_j v_ij . grad_i W(h_i),
 *               curl_i = |(1/rho_i) sum_j m_j v_ij x grad_i W(h_i)|, and
 *               Balsara's factor f_i = |div_i| / (|div_i| + curl_i + 1e-4 c_i/h_i)
 *               multiplying Pi_ij by (f_i + f_j)/2.
 *   conduction  (optional) over the force pair set, with conductivity kappa
 *               per particle (heat flux -kappa grad u):
 *               du_i^cond = sum_j m_j/(rho_i rho_j) 4 kappa_i kappa_j/(kappa_i + kappa_j)
 *                           (u_i - u_j) Fbar_ij,  Fbar_ij = (F(h_i) + F(h_j))/2,
 *               F(h) = dW/dr(r_ij, h) / r_ij.
 *   gravity     (separate pass) short-range TreePM gravity by a Barnes-Hut
 *               walk over a tree fixed by definition; see orc_gravity.
 *
 * Everything is a direct sum in FP64 over an explicit candidate set: either
 * every particle (brute force) or the particles of the cells around i in a
 * Morton-ordered cell list (a plain lower_bound per cell). No blocking, no
 * reordering of the arithmetic.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_TWO32 4294967296.0
#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* Quantisation and Morton keys                                              */
/* ------------------------------------------------------------------------- */

/* X = rint(frac(x/L) * 2^32) mod 2^32; rint rounds half to even. */
void orc_quantize(const double *pos, int64_t n3, double L, uint32_t *X)
{
    for (int64_t k = 0; k < n3; ++k) {
        double t = pos[k] / L;
        t = t - floor(t);
        double v = rint(t * ORC_TWO32);
        if (v >= ORC_TWO32) v -= ORC_TWO32;
        X[k] = (uint32_t)(uint64_t)v;
    }
}

/* Spread the low 21 bits of v so that bit b lands at bit 3b. Written as a
 * loop over bits, the plainest possible form. */
static uint64_t orc_spread3(uint32_t v)
{
    uint64_t r = 0;
    for (int b = 0; b < 21; ++b)
        r |= (uint64_t)((v >> b) & 1u) << (3 * b);
    return r;
}

/* 63-bit Morton key of the top 21 bits of each axis; within each bit triple x
 * is the most significant, then y, then z. */
uint64_t orc_morton(uint32_t X, uint32_t Y, uint32_t Z)
{
    return (orc_spread3(X >> 11) << 2) | (orc_spread3(Y >> 11) << 1) | orc_spread3(Z >> 11);
}

/* Keys of a batch of boxes: box b in the top bb bits, the Morton key shifted
 * down by bb bits below it (bb = ceil(log2(n_boxes)), 0 for one box). */
void orc_keys(const uint32_t *X, int64_t n, int64_t box, int bb, uint64_t *key)
{
    for (int64_t i = 0; i < n; ++i) {
        uint64_t m = orc_morton(X[3 * i], X[3 * i + 1], X[3 * i + 2]);
        key[i] = bb ? (((uint64_t)box << (63 - bb)) | (m >> bb)) : m;
    }
}

typedef struct { uint64_t key; int64_t idx; } orc_ki;

static int orc_ki_cmp(const void *a, const void *b)
{
    const orc_ki *x = (const orc_ki *)a, *y = (const orc_ki *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/* Sort (key, index) by key, ties by index; writes the permutation. */
void orc_sort_keys(const uint64_t *key, int64_t n, int64_t *perm)
{
    orc_ki *a = (orc_ki *)malloc(sizeof(orc_ki) * (size_t)(n ? n : 1));
    for (int64_t i = 0; i < n; ++i) { a[i].key = key[i]; a[i].idx = i; }
    qsort(a, (size_t)n, sizeof(orc_ki), orc_ki_cmp);
    for (int64_t i = 0; i < n; ++i) perm[i] = a[i].idx;
    free(a);
}

/* ------------------------------------------------------------------------- */
/* Kernel                                                                    */
/* ------------------------------------------------------------------------- */

double orc_w(double q)
{
    if (q < 0.0) q = -q;
    if (q <= 0.5) return 1.0 - 6.0 * q * q + 6.0 * q * q * q;
    if (q < 1.0) { double a = 1.0 - q; return 2.0 * a * a * a; }
    return 0.0;
}

double orc_dw(double q) /* dw/dq */
{
    if (q <= 0.5) return -12.0 * q + 18.0 * q * q;
    if (q < 1.0) { double a = 1.0 - q; return -6.0 * a * a; }
    return 0.0;
}

double orc_W(double r, double h) { return 8.0 / (ORC_PI * h * h * h) * orc_w(r / h); }
double orc_dWdr(double r, double h) { return 8.0 / (ORC_PI * h * h * h * h) * orc_dw(r / h); }
double orc_dWdh(double r, double h) { return -(3.0 * orc_W(r, h) + r * orc_dWdr(r, h)) / h; }

/* ------------------------------------------------------------------------- */
/* Particle positions: quantised (exact integer geometry) or continuous      */
/* ------------------------------------------------------------------------- */

typedef struct {
    int mode;            /* 0: quantised X, 1: continuous FP64 positions */
    const uint32_t *X;   /* n x 3, always present (continuous mode: for indexing) */
    const double *xc;    /* n x 3, continuous mode only */
    int64_t n;
    double L;
} orc_pos;

/* Separation vector r_ij = x_i - x_j (physical units, minimum image) and the
 * neighbour predicate "r < h" evaluated as the contract states. */
static int orc_pair(const orc_pos *P, int64_t i, int64_t j, double h, double rij[3], double *r)
{
    if (P->mode == 0) {
        const uint32_t *a = P->X + 3 * i, *b = P->X + 3 * j;
        uint64_t D2 = 0;
        for (int k = 0; k < 3; ++k) {
            int32_t d = (int32_t)(a[k] - b[k]);
            int64_t dd = d;
            D2 += (uint64_t)(dd * dd);
            rij[k] = (double)d * (P->L / ORC_TWO32);
        }
        double H = h * ORC_TWO32 / P->L;
        *r = sqrt((double)D2) * (P->L / ORC_TWO32);
        return (double)D2 < H * H;
    } else {
        const double *a = P->xc + 3 * i, *b = P->xc + 3 * j;
        double r2 = 0.0;
        for (int k = 0; k < 3; ++k) {
            double d = a[k] - b[k];
            d -= P->L * rint(d / P->L);
            rij[k] = d;
            r2 += d * d;
        }
        *r = sqrt(r2);
        return r2 < h * h;
    }
}

/* ------------------------------------------------------------------------- */
/* Morton cell list                                                          */
/* ------------------------------------------------------------------------- */

typedef struct {
    int64_t n;
    uint64_t *key;   /* sorted keys */
    int64_t *idx;    /* particle index of each sorted key */
} orc_index;

void *orc_index_new(const uint32_t *X, int64_t n)
{
    orc_index *I = (orc_index *)calloc(1, sizeof(orc_index));
    I->n = n;
    uint64_t *k = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n ? n : 1));
    I->key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n ? n : 1));
    I->idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    orc_keys(X, n, 0, 0, k);
    orc_sort_keys(k, n, I->idx);
    for (int64_t s = 0; s < n; ++s) I->key[s] = k[I->idx[s]];
    free(k);
    return I;
}

void orc_index_free(void *p)
{
    orc_index *I = (orc_index *)p;
    if (!I) return;
    free(I->key); free(I->idx); free(I);
}

static int64_t orc_lower_bound(const uint64_t *a, int64_t n, uint64_t v)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

typedef struct { int64_t *a; int64_t n, cap; } orc_buf;

static void orc_push(orc_buf *b, int64_t v)
{
    if (b->n == b->cap) {
        b->cap = b->cap ? 2 * b->cap : 1024;
        b->a = (int64_t *)realloc(b->a, sizeof(int64_t) * (size_t)b->cap);
    }
    b->a[b->n++] = v;
}

/* Candidates for a sphere of radius H (integer units) around integer point
 * C: every particle of the cells, at the finest level whose cell side is at
 * least H, that touch the 3x3x3 block around C's cell (periodic). The caller
 * applies the exact predicate. Requires H <= 2^31. */
static void orc_candidates(const orc_index *I, const uint32_t C[3], double H, orc_buf *out)
{
    out->n = 0;
    int lvl = 21;
    while (lvl > 1 && ldexp(1.0, 32 - lvl) < H) --lvl;
    uint32_t ncell = 1u << lvl;
    int shift = 32 - lvl;
    uint32_t c[3];
    for (int k = 0; k < 3; ++k) c[k] = C[k] >> shift;
    uint32_t seen[27][3];
    int nseen = 0;
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
                uint32_t cc[3] = {(c[0] + ncell + (uint32_t)dx) % ncell,
                                  (c[1] + ncell + (uint32_t)dy) % ncell,
                                  (c[2] + ncell + (uint32_t)dz) % ncell};
                int dup = 0;
                for (int s = 0; s < nseen; ++s)
                    if (seen[s][0] == cc[0] && seen[s][1] == cc[1] && seen[s][2] == cc[2]) dup = 1;
                if (dup) continue;
                memcpy(seen[nseen++], cc, sizeof cc);
                /* cell cc at level lvl covers keys [p << 3(21-lvl), (p+1) << 3(21-lvl)) */
                uint64_t p = (orc_spread3(cc[0]) << 2) | (orc_spread3(cc[1]) << 1) | orc_spread3(cc[2]);
                int sh = 3 * (21 - lvl);
                uint64_t k0 = p << sh, k1 = (p + 1) << sh;
                int64_t s0 = orc_lower_bound(I->key, I->n, k0);
                int64_t s1 = orc_lower_bound(I->key, I->n, k1);
                for (int64_t s = s0; s < s1; ++s) orc_push(out, I->idx[s]);
            }
}

/* Candidate set for particle i: brute force (all particles) or cell list. */
static void orc_cands_for(const orc_pos *P, const orc_index *I, int64_t i, double h, orc_buf *out)
{
    if (!I) {
        out->n = 0;
        for (int64_t j = 0; j < P->n; ++j) orc_push(out, j);
        return;
    }
    /* Integer radius with a margin that covers the continuous-mode
     * quantisation of the indexed positions (<= 1 unit per axis). */
    double H = h * ORC_TWO32 / P->L * (1.0 + 1e-12) + 4.0;
    orc_candidates(I, P->X + 3 * i, H, out);
}

/* Index offset of the neighbour-set checksums (test instrumentation: a box
 * checked on its own whose particles sit at an offset in a batch). */
static int64_t orc_hash_off = 0;
void orc_set_hash_offset(int64_t off) { orc_hash_off = off; }

/* splitmix64 finaliser (Steele, Lea, Flood 2014): order-independent
 * neighbour-set checksum = sum over the set of splitmix64(index). */
uint64_t orc_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* ------------------------------------------------------------------------- */
/* Density                                                                   */
/* ------------------------------------------------------------------------- */

typedef struct {
    double neff, dneff, rho, drho;
    int64_t nngb;
    uint64_t hash;
} orc_dens;

static void orc_density_at(const orc_pos *P, const orc_index *I, const double *m, int64_t i,
                           double h, orc_buf *cb, orc_dens *o)
{
    orc_cands_for(P, I, i, h, cb);
    double sw = 0.0, sdw = 0.0, rho = 0.0, drho = 0.0;
    int64_t nn = 0;
    uint64_t hs = 0;
    for (int64_t c = 0; c < cb->n; ++c) {
        int64_t j = cb->a[c];
        double rij[3], r;
        int in = orc_pair(P, i, j, h, rij, &r);
        if (j == i) { r = 0.0; in = 1; }
        if (!in) continue;
        double W = orc_W(r, h);
        sw += W;
        sdw += orc_dWdh(r, h);
        rho += m[j] * W;
        drho += m[j] * orc_dWdh(r, h);
        if (j != i) { ++nn; hs += orc_splitmix64((uint64_t)(j + orc_hash_off)); }
    }
    double f = 4.0 * ORC_PI / 3.0 * h * h * h;
    o->neff = f * sw;
    /* d/dh [ (4pi/3) h^3 sum W ] */
    o->dneff = 4.0 * ORC_PI * h * h * sw + f * sdw;
    o->rho = rho;
    o->drho = drho;
    o->nngb = nn;
    o->hash = hs;
}

/* Status bits per particle. */
#define ORC_NOT_CONVERGED 1
#define ORC_H_TOO_LARGE 2

/*
 * Density pass for the active particles (NULL = all). fixed_h != 0 evaluates
 * at h_init without iterating. Otherwise h solves N_eff(h) = n_target to
 * |N_eff - n_target| <= tol, starting from h_init[i] (<= 0: from a small
 * global guess grown by factors of 2 until the root is bracketed), with a
 * Newton step whenever it stays inside the bracket and bisection otherwise.
 * Outputs are indexed by particle. Returns the OR of the status bits.
 */
int orc_density(int mode, const uint32_t *X, const double *xc, int64_t n, double L,
                const double *m, const double *h_init, double n_target, double tol,
                int max_iter, const int64_t *active, int64_t n_active, int brute, int fixed_h,
                double *h_out, double *rho, double *drho_dh, double *omega, double *neff,
                int64_t *n_ngb, uint64_t *hash, int32_t *status)
{
    orc_pos P = {mode, X, xc, n, L};
    orc_index *I = brute ? NULL : (orc_index *)orc_index_new(X, n);
    int64_t na = active ? n_active : n;
    double h_glob = L * cbrt(3.0 * n_target / (4.0 * ORC_PI * (double)n));
    double h_cap = 0.5 * L * (1.0 - 1e-9); /* h must stay below L/2 */
    int any = 0;
#pragma omp parallel reduction(| : any)
    {
        orc_buf cb = {0, 0, 0};
#pragma omp for schedule(dynamic, 16)
        for (int64_t a = 0; a < na; ++a) {
            int64_t i = active ? active[a] : a;
            int st = 0;
            orc_dens d;
            double h = (h_init && h_init[i] > 0.0) ? h_init[i] : h_glob / 64.0;
            if (h >= h_cap) h = 0.5 * h_cap;
            orc_density_at(&P, I, m, i, h, &cb, &d);
            if (!fixed_h) {
                double lo = 0.0, hi = INFINITY;
                int it = 0;
                while (fabs(d.neff - n_target) > tol) {
                    if (++it > max_iter) { st |= ORC_NOT_CONVERGED; break; }
                    if (d.neff < n_target) lo = h; else hi = h;
                    double hn;
                    if (isinf(hi)) {
                        /* not bracketed yet: grow (Newton if it grows by less) */
                        if (h >= h_cap) { st |= ORC_H_TOO_LARGE; break; }
                        hn = 2.0 * h;
                        if (d.dneff > 0.0) {
                            double hnewt = h - (d.neff - n_target) / d.dneff;
                            if (hnewt > h && hnewt < hn) hn = hnewt;
                        }
                        if (hn >= h_cap) hn = h_cap;
                    } else {
                        hn = (d.dneff > 0.0) ? h - (d.neff - n_target) / d.dneff : NAN;
                        if (!(hn > lo && hn < hi)) hn = 0.5 * (lo + hi);
                    }
                    h = hn;
                    orc_density_at(&P, I, m, i, h, &cb, &d);
                }
            }
            h_out[i] = h;
            rho[i] = d.rho;
            drho_dh[i] = d.drho;
            omega[i] = 1.0 / (1.0 + h / (3.0 * d.rho) * d.drho);
            if (neff) neff[i] = d.neff;
            n_ngb[i] = d.nngb;
            if (hash) hash[i] = d.hash;
            if (status) status[i] = st;
            any |= st;
        }
        free(cb.a);
    }
    orc_index_free(I);
    return any;
}

/* ------------------------------------------------------------------------- */
/* Force                                                                     */
/* ------------------------------------------------------------------------- */

/* Morton cell lists of the particles grouped by smoothing-length level: level
 * l holds the particles whose h fits one level-l cell (2^-l L >= h > 2^-l-1 L),
 * so every j with r_ij < h_j lies in the 3x3x3 level-l cells around i. This
 * finds the half of the symmetric pair set that i's own radius misses. */
typedef struct {
    orc_index *lv[22];
    int64_t *map[22];   /* local index -> particle index */
} orc_hindex;

static int orc_hlevel(double h, double L)
{
    /* finest level whose cell side (integer units) exceeds H + 4 units */
    double H = h * ORC_TWO32 / L + 4.0;
    int l = 21;
    while (l > 1 && ldexp(1.0, 32 - l) < H) --l;
    return l;
}

static orc_hindex *orc_hindex_new(const orc_pos *P, const double *h)
{
    orc_hindex *Hx = (orc_hindex *)calloc(1, sizeof(orc_hindex));
    int64_t cnt[22] = {0};
    for (int64_t j = 0; j < P->n; ++j) cnt[orc_hlevel(h[j], P->L)]++;
    for (int l = 0; l < 22; ++l) {
        if (!cnt[l]) continue;
        uint32_t *Xl = (uint32_t *)malloc(sizeof(uint32_t) * 3 * (size_t)cnt[l]);
        Hx->map[l] = (int64_t *)malloc(sizeof(int64_t) * (size_t)cnt[l]);
        int64_t k = 0;
        for (int64_t j = 0; j < P->n; ++j)
            if (orc_hlevel(h[j], P->L) == l) {
                memcpy(Xl + 3 * k, P->X + 3 * j, 3 * sizeof(uint32_t));
                Hx->map[l][k++] = j;
            }
        Hx->lv[l] = (orc_index *)orc_index_new(Xl, cnt[l]);
        free(Xl);
    }
    return Hx;
}

static void orc_hindex_free(orc_hindex *Hx)
{
    if (!Hx) return;
    for (int l = 0; l < 22; ++l) { orc_index_free(Hx->lv[l]); free(Hx->map[l]); }
    free(Hx);
}

/*
 * Velocity divergence and curl of the active particles (NULL = all) at the
 * given h and rho (the density pass's): over j != i with r_ij < h_i,
 *   div_i  = -(1/rho_i) sum_j m_j v_ij . grad_i W_ij(h_i)
 *   curl_i = |(1/rho_i) sum_j m_j v_ij x grad_i W_ij(h_i)|
 * with v_ij = v_i - v_j, r_ij = x_i - x_j, grad_i W_ij = dW/dr(r_ij, h_i)
 * r_ij / |r_ij| (coincident pairs add nothing). These are the SPH estimates
 * of the velocity gradient that Gadget-2 forms in its density loop for the
 * Balsara switch; the paper's code runs an "improved SPH" of this lineage
 * (Sec. 1). scale_d / scale_c (optional): (1/rho_i) sum_j of the magnitudes
 * of the pair terms of the divergence and of the curl vector (per-particle
 * absolute scales for tolerances).
 */
void orc_divcurl(int mode, const uint32_t *X, const double *xc, int64_t n, double L,
                 const double *v, const double *m, const double *h, const double *rho,
                 const int64_t *active, int64_t n_active, int brute, double *divv, double *curlv,
                 double *scale_d, double *scale_c)
{
    orc_pos P = {mode, X, xc, n, L};
    orc_index *I = brute ? NULL : (orc_index *)orc_index_new(X, n);
    int64_t na = active ? n_active : n;
#pragma omp parallel
    {
        orc_buf cb = {0, 0, 0};
#pragma omp for schedule(dynamic, 16)
        for (int64_t a = 0; a < na; ++a) {
            int64_t i = active ? active[a] : a;
            orc_cands_for(&P, I, i, h[i], &cb);
            double sd = 0.0, sc[3] = {0.0, 0.0, 0.0}, ad = 0.0, ac = 0.0;
            for (int64_t c = 0; c < cb.n; ++c) {
                int64_t j = cb.a[c];
                if (j == i) continue;
                double rij[3], r;
                if (!orc_pair(&P, i, j, h[i], rij, &r) || r == 0.0) continue;
                double g = m[j] * orc_dWdr(r, h[i]) / r;   /* m_j grad_i W = g * r_ij */
                double vij[3] = {v[3 * i] - v[3 * j], v[3 * i + 1] - v[3 * j + 1], v[3 * i + 2] - v[3 * j + 2]};
                double td = g * (vij[0] * rij[0] + vij[1] * rij[1] + vij[2] * rij[2]);
                double tc[3] = {g * (vij[1] * rij[2] - vij[2] * rij[1]), g * (vij[2] * rij[0] - vij[0] * rij[2]),
                                g * (vij[0] * rij[1] - vij[1] * rij[0])};
                sd += td;
                sc[0] += tc[0];
                sc[1] += tc[1];
                sc[2] += tc[2];
                ad += fabs(td);
                ac += sqrt(tc[0] * tc[0] + tc[1] * tc[1] + tc[2] * tc[2]);
            }
            divv[i] = -sd / rho[i];
            curlv[i] = sqrt(sc[0] * sc[0] + sc[1] * sc[1] + sc[2] * sc[2]) / rho[i];
            if (scale_d) scale_d[i] = ad / rho[i];
            if (scale_c) scale_c[i] = ac / rho[i];
        }
        free(cb.a);
    }
    orc_index_free(I);
}

/* Balsara's viscosity limiter from div v, |curl v|, sound speed and h. */
static double orc_balsara(double div, double curl, double cs, double h)
{
    double ad = fabs(div);
    return ad / (ad + curl + 1e-4 * cs / h);
}

/*
 * Hydro-force pass for the active particles (NULL = all). Inputs are indexed
 * by particle (all n, neighbours included). Outputs, for active i only:
 * acc (n x 3), dudt, vsig; scale_a / scale_u = sum over pairs of the
 * magnitude of each pair's term (the per-particle absolute scale used for
 * tolerances); n_pairs = |pair set|; hash = neighbour-set checksum.
 * divv / curlv (both NULL or both given): Balsara's switch on Pi_ij.
 * alpha_p (NULL: alpha for every pair): a viscosity parameter per particle,
 * the pair taking alpha_ij = (alpha_i + alpha_j) / 2 (time-dependent
 * viscosity, Morris & Monaghan 1997), symmetric in i and j.
 */
void orc_force(int mode, const uint32_t *X, const double *xc, int64_t n, double L,
               const double *v, const double *m, const double *u, const double *h,
               const double *rho, const double *omega, double alpha, const double *alpha_p, double gamma,
               const double *divv, const double *curlv,
               const int64_t *active, int64_t n_active, int brute,
               double *acc, double *dudt, double *vsig, double *scale_a, double *scale_u,
               int64_t *n_pairs, uint64_t *hash)
{
    orc_pos P = {mode, X, xc, n, L};
    orc_index *I = brute ? NULL : (orc_index *)orc_index_new(X, n);
    orc_hindex *Hx = brute ? NULL : orc_hindex_new(&P, h);
    int64_t na = active ? n_active : n;
#pragma omp parallel
    {
        orc_buf cb = {0, 0, 0}, cl = {0, 0, 0};
#pragma omp for schedule(dynamic, 16)
        for (int64_t a = 0; a < na; ++a) {
            int64_t i = active ? active[a] : a;
            /* Candidates: i's own sphere, plus (cell-list mode) every level's
             * 3x3x3 block for the particles whose own sphere reaches i. Each j
             * is taken once: from the first list if r < h_i, else from its
             * level list if r < h_j. */
            orc_cands_for(&P, I, i, h[i], &cb);
            int64_t nfirst = cb.n;
            if (Hx) {
                for (int l = 0; l < 22; ++l) {
                    if (!Hx->lv[l]) continue;
                    orc_candidates(Hx->lv[l], X + 3 * i, ldexp(1.0, 32 - l), &cl);
                    for (int64_t c = 0; c < cl.n; ++c) orc_push(&cb, Hx->map[l][cl.a[c]]);
                }
            }
            double Pi = (gamma - 1.0) * rho[i] * u[i];
            double ci = sqrt(gamma * Pi / rho[i]);
            double Ai = omega[i] * Pi / (rho[i] * rho[i]);
            double fi = divv ? orc_balsara(divv[i], curlv[i], ci, h[i]) : 1.0;
            double ax = 0, ay = 0, az = 0, du = 0, vs = 0.0, sa = 0.0, su = 0.0;
            int64_t np = 0;
            uint64_t hs = 0;
            for (int64_t c = 0; c < cb.n; ++c) {
                int64_t j = cb.a[c];
                if (j == i) continue;
                double rij[3], r;
                int in_i = orc_pair(&P, i, j, h[i], rij, &r);
                int in_j = orc_pair(&P, i, j, h[j], rij, &r);
                int take;
                if (!Hx) take = in_i || in_j;          /* brute force: every j once */
                else if (c < nfirst) take = in_i;      /* i's own sphere */
                else take = !in_i && in_j;             /* j's sphere only */
                if (!take) continue;
                ++np;
                hs += orc_splitmix64((uint64_t)(j + orc_hash_off));
                double Pj = (gamma - 1.0) * rho[j] * u[j];
                double cj = sqrt(gamma * Pj / rho[j]);
                double Aj = omega[j] * Pj / (rho[j] * rho[j]);
                double vij[3] = {v[3 * i] - v[3 * j], v[3 * i + 1] - v[3 * j + 1], v[3 * i + 2] - v[3 * j + 2]};
                if (r == 0.0) {
                    /* coincident: no direction, all pair terms vanish */
                    double vsg = ci + cj;
                    if (vsg > vs) vs = vsg;
                    continue;
                }
                double vr = vij[0] * rij[0] + vij[1] * rij[1] + vij[2] * rij[2];
                double wij = vr / r;
                double vsg = ci + cj - 3.0 * wij;
                if (vsg > vs) vs = vsg;
                double Fi = orc_dWdr(r, h[i]) / r; /* grad_i W(h_i) = Fi * r_ij */
                double Fj = orc_dWdr(r, h[j]) / r;
                double Fbar = 0.5 * (Fi + Fj);
                double PIij = 0.0;
                double aij = alpha_p ? 0.5 * (alpha_p[i] + alpha_p[j]) : alpha;
                if (wij < 0.0) PIij = -0.5 * aij * vsg * wij / (0.5 * (rho[i] + rho[j]));
                if (divv) PIij *= 0.5 * (fi + orc_balsara(divv[j], curlv[j], cj, h[j]));
                double coef = m[j] * (Ai * Fi + Aj * Fj + PIij * Fbar);
                ax -= coef * rij[0];
                ay -= coef * rij[1];
                az -= coef * rij[2];
                double dut = m[j] * (Ai * Fi * vr + 0.5 * PIij * Fbar * vr);
                du += dut;
                sa += fabs(coef) * r;
                su += fabs(dut);
            }
            acc[3 * i] = ax; acc[3 * i + 1] = ay; acc[3 * i + 2] = az;
            dudt[i] = du;
            vsig[i] = vs;
            if (scale_a) scale_a[i] = sa;
            if (scale_u) scale_u[i] = su;
            if (n_pairs) n_pairs[i] = np;
            if (hash) hash[i] = hs;
        }
        free(cb.a);
        free(cl.a);
    }
    orc_hindex_free(Hx);
    orc_index_free(I);
}

/*
 * Thermal conduction heating rate of the active particles (NULL = all) over
 * the force pass's pair set (j != i, r_ij < max(h_i, h_j)). The paper's code
 * has a conduction module (Sec. 1); the paper states no formula, so this is
 * the SPH conduction form of Cleary & Monaghan (1999), as Jubelgas, Springel &
 * Dolag (2004) used it in Gadget, written for u with a conductivity kappa per
 * particle (heat flux -kappa grad u):
 *   du_i = sum_j m_j / (rho_i rho_j) * 4 kappa_i kappa_j / (kappa_i + kappa_j)
 *          * (u_i - u_j) * Fbar_ij,
 *   Fbar_ij = (F(r_ij, h_i) + F(r_ij, h_j)) / 2,  F(r, h) = dW/dr(r, h) / r,
 * a pair term antisymmetric in i and j (sum_i m_i du_i = 0). The harmonic
 * mean is 0 when either kappa is 0; coincident pairs add nothing.
 * scale (optional): sum over pairs of the magnitudes of the terms.
 */
void orc_conduction(int mode, const uint32_t *X, const double *xc, int64_t n, double L,
                    const double *m, const double *u, const double *h, const double *rho,
                    const double *kappa, const int64_t *active, int64_t n_active, int brute,
                    double *dudt, double *scale)
{
    orc_pos P = {mode, X, xc, n, L};
    orc_index *I = brute ? NULL : (orc_index *)orc_index_new(X, n);
    orc_hindex *Hx = brute ? NULL : orc_hindex_new(&P, h);
    int64_t na = active ? n_active : n;
#pragma omp parallel
    {
        orc_buf cb = {0, 0, 0}, cl = {0, 0, 0};
#pragma omp for schedule(dynamic, 16)
        for (int64_t a = 0; a < na; ++a) {
            int64_t i = active ? active[a] : a;
            /* the force pass's candidates: i's own sphere, then the level lists */
            orc_cands_for(&P, I, i, h[i], &cb);
            int64_t nfirst = cb.n;
            if (Hx) {
                for (int l = 0; l < 22; ++l) {
                    if (!Hx->lv[l]) continue;
                    orc_candidates(Hx->lv[l], X + 3 * i, ldexp(1.0, 32 - l), &cl);
                    for (int64_t c = 0; c < cl.n; ++c) orc_push(&cb, Hx->map[l][cl.a[c]]);
                }
            }
            double du = 0.0, sc = 0.0;
            for (int64_t c = 0; c < cb.n; ++c) {
                int64_t j = cb.a[c];
                if (j == i) continue;
                double rij[3], r;
                int in_i = orc_pair(&P, i, j, h[i], rij, &r);
                int in_j = orc_pair(&P, i, j, h[j], rij, &r);
                int take;
                if (!Hx) take = in_i || in_j;
                else if (c < nfirst) take = in_i;
                else take = !in_i && in_j;
                if (!take || r == 0.0) continue;
                double ks = kappa[i] + kappa[j];
                double kij = ks > 0.0 ? 4.0 * kappa[i] * kappa[j] / ks : 0.0;
                double Fbar = 0.5 * (orc_dWdr(r, h[i]) + orc_dWdr(r, h[j])) / r;
                double t = m[j] / (rho[i] * rho[j]) * kij * (u[i] - u[j]) * Fbar;
                du += t;
                sc += fabs(t);
            }
            dudt[i] = du;
            if (scale) scale[i] = sc;
        }
        free(cb.a);
        free(cl.a);
    }
    orc_hindex_free(Hx);
    orc_index_free(I);
}

/* Brute-force neighbour list of one particle at radius h (for pins). */
int64_t orc_neighbours(int mode, const uint32_t *X, const double *xc, int64_t n, double L,
                       int64_t i, double h, int brute, int64_t *out, int64_t cap)
{
    orc_pos P = {mode, X, xc, n, L};
    orc_index *I = brute ? NULL : (orc_index *)orc_index_new(X, n);
    orc_buf cb = {0, 0, 0};
    orc_cands_for(&P, I, i, h, &cb);
    int64_t k = 0;
    for (int64_t c = 0; c < cb.n; ++c) {
        int64_t j = cb.a[c];
        double rij[3], r;
        if (j == i) continue;
        if (orc_pair(&P, i, j, h, rij, &r)) { if (k < cap) out[k] = j; ++k; }
    }
    free(cb.a);
    orc_index_free(I);
    return k;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the following parallel regions (the 1-core timing of the CPU
 * baseline); returns the previous count. */
int orc_set_threads(int t)
{
    int old = orc_num_threads();
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#endif
    return old;
}

/* Vectorised kernel evaluation for the pins (w, dw/dq at each q). */
void orc_kernel_array(const double *q, int64_t n, double *w, double *dw)
{
    for (int64_t k = 0; k < n; ++k) { w[k] = orc_w(q[k]); dw[k] = orc_dw(q[k]); }
}

/*
 * Symmetric pair set of the force pass: every ordered pair (i, j), i != j,
 * with r_ij < max(h_i, h_j) under the contract's predicate, found by brute
 * force (all j) or the two cell lists of orc_force. Writes up to cap pairs
 * into out_i/out_j, returns the total count (call again with a larger cap if
 * it exceeds cap). Serial, in order of i then candidate order.
 */
int64_t orc_pair_list(int mode, const uint32_t *X, const double *xc, int64_t n, double L,
                      const double *h, int brute, int64_t *out_i, int64_t *out_j, int64_t cap)
{
    orc_pos P = {mode, X, xc, n, L};
    orc_index *I = brute ? NULL : (orc_index *)orc_index_new(X, n);
    orc_hindex *Hx = brute ? NULL : orc_hindex_new(&P, h);
    orc_buf cb = {0, 0, 0}, cl = {0, 0, 0};
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        orc_cands_for(&P, I, i, h[i], &cb);
        int64_t nfirst = cb.n;
        if (Hx) {
            for (int l = 0; l < 22; ++l) {
                if (!Hx->lv[l]) continue;
                orc_candidates(Hx->lv[l], X + 3 * i, ldexp(1.0, 32 - l), &cl);
                for (int64_t c = 0; c < cl.n; ++c) orc_push(&cb, Hx->map[l][cl.a[c]]);
            }
        }
        for (int64_t c = 0; c < cb.n; ++c) {
            int64_t j = cb.a[c];
            if (j == i) continue;
            double rij[3], r;
            int in_i = orc_pair(&P, i, j, h[i], rij, &r);
            int in_j = orc_pair(&P, i, j, h[j], rij, &r);
            int take;
            if (!Hx) take = in_i || in_j;
            else if (c < nfirst) take = in_i;
            else take = !in_i && in_j;
            if (!take) continue;
            if (k < cap) { out_i[k] = i; out_j[k] = j; }
            ++k;
        }
    }
    free(cb.a);
    free(cl.a);
    orc_hindex_free(Hx);
    orc_index_free(I);
    return k;
}

/* ------------------------------------------------------------------------- */
/* Gravity: short-range part of the TreePM split by a Barnes-Hut walk        */
/* ------------------------------------------------------------------------- */

/*
 * The paper's code computes short-range gravity by Barnes-Hut (particles
 * interact with distant tree nodes as point masses, chosen by an opening
 * criterion; the interactions happen inside the walk) and long-range gravity
 * by a particle mesh (Sec. 1, Sec. 3). This is the short-range part, in the
 * form of Gadget's TreePM split (Springel 2005), on a tree fixed by
 * definition so that the approximation itself is reproducible:
 *
 *   tree     particles sorted by Morton key (ties by index); a leaf is 8
 *            consecutive sorted particles, a level-k node is 8 consecutive
 *            level-(k-1) nodes, up to a single root. A node's box is the
 *            min/max of its particles' integer coordinates, its mass and
 *            centre of mass the plain sums.
 *   decisions in coarse integer units (integer coordinates >> 8, i.e.
 *            2^-24 L): for particle i and a node, G_a = periodic gap between
 *            X_i and the node's box on axis a, D2 = sum G_a^2, l = largest side,
 *            L2 = l^2; F2 = sum of the squared far distances to the box,
 *            F_a = (periodic distance from X_i to the far side of the box +
 *            255) >> 8 (rounded up). All tests are integer comparisons:
 *            RCi = ceil((r_cut 2^24 / L)^2) (FP64, then exact), so that
 *            "D2 < RCi" is "coarse distance below r_cut"; the opening angle
 *            enters as P = rint(theta^2 2^16). The root is always opened. A
 *            child of an opened node is
 *              skipped   if D2 >= RCi (the box lies beyond the cutoff),
 *              accepted  (monopole) if P > 0, D2 > 0, F2 < RCi (the box lies
 *                        inside the cutoff, so that every member would
 *                        interact), L2 <= D2 and 2^16 L2 <= P D2 (opening
 *                        angle: l <= theta D),
 *              opened    otherwise (a leaf: its particles one by one).
 *            A particle j != i of an opened leaf interacts if its coarse
 *            distance, sum_a (|(int32)(X_j - X_i)| >> 8)^2, is below RCi.
 *   pair     a_i += G m_j K(r) (x_j - x_i), minimum image, with
 *            K(r) = M(r/h_s) / r^3 * g(r): M the mass fraction of the cubic
 *            spline of support h_s inside r (1 for r >= h_s; Gadget's
 *            softening), g(r) = erfc(r / (2 r_s)) + r / (r_s sqrt(pi))
 *            exp(-r^2 / (4 r_s^2)) the short-range factor (1 without a
 *            split, r_s <= 0). A node acts as its mass at its centre of mass.
 *            Coincident pairs (r = 0) exert nothing.
 */

/* Fraction of a cubic-spline (support 1) mass inside radius q:
 * 32 int_0^q w(s) s^2 ds, piece by piece. */
double orc_soft_mass(double q)
{
    if (q >= 1.0) return 1.0;
    double a = q < 0.5 ? q : 0.5;
    double inner = a * a * a / 3.0 - 6.0 * pow(a, 5) / 5.0 + pow(a, 6);
    if (q <= 0.5) return 32.0 * inner;
#define ORC_F2(s) (2.0 * ((s) * (s) * (s) / 3.0 - 3.0 * pow((s), 4) / 4.0 + 3.0 * pow((s), 5) / 5.0 - pow((s), 6) / 6.0))
    double outer = ORC_F2(q) - ORC_F2(0.5);
#undef ORC_F2
    return 32.0 * (inner + outer);
}

/* K(r): the acceleration per unit mass and unit separation vector. */
static double orc_grav_K(double r, double hs, double rs)
{
    double Mq = hs > 0.0 ? orc_soft_mass(r / hs) : 1.0;
    double g = 1.0;
    if (rs > 0.0) g = erfc(r / (2.0 * rs)) + r / (rs * sqrt(ORC_PI)) * exp(-r * r / (4.0 * rs * rs));
    return Mq / (r * r * r) * g;
}

typedef struct {
    int nlev;
    int64_t cnt[32], off[32];   /* nodes per level, first node of the level */
    uint32_t *lo, *hi;          /* 3 per node */
    double *mass, *com;         /* com: 3 per node, integer units */
} orc_tree;

static void orc_tree_build(const uint32_t *X, const double *m, const int64_t *sorted, int64_t n, orc_tree *T)
{
    int64_t c = (n + 7) / 8, total = 0;
    T->nlev = 0;
    for (;;) {
        T->cnt[T->nlev] = c;
        T->off[T->nlev] = total;
        total += c;
        T->nlev++;
        if (c == 1) break;
        c = (c + 7) / 8;
    }
    T->lo = (uint32_t *)malloc(sizeof(uint32_t) * 3 * total);
    T->hi = (uint32_t *)malloc(sizeof(uint32_t) * 3 * total);
    T->mass = (double *)malloc(sizeof(double) * total);
    T->com = (double *)malloc(sizeof(double) * 3 * total);
    for (int k = 0; k < T->nlev; ++k) {
        for (int64_t t = 0; t < T->cnt[k]; ++t) {
            int64_t nd = T->off[k] + t;
            uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0, 0, 0};
            double M = 0.0, S[3] = {0.0, 0.0, 0.0};
            /* members: particles (leaf) or child nodes */
            int64_t a = 8 * t, b = a + 8, lim = k == 0 ? n : T->cnt[k - 1];
            if (b > lim) b = lim;
            for (int64_t e = a; e < b; ++e) {
                for (int d = 0; d < 3; ++d) {
                    uint32_t l, h;
                    if (k == 0) {
                        l = h = X[3 * sorted[e] + d];
                    } else {
                        l = T->lo[3 * (T->off[k - 1] + e) + d];
                        h = T->hi[3 * (T->off[k - 1] + e) + d];
                    }
                    if (l < lo[d]) lo[d] = l;
                    if (h > hi[d]) hi[d] = h;
                }
                double me = k == 0 ? m[sorted[e]] : T->mass[T->off[k - 1] + e];
                for (int d = 0; d < 3; ++d) {
                    double xe = k == 0 ? (double)X[3 * sorted[e] + d] : T->com[3 * (T->off[k - 1] + e) + d];
                    S[d] += me * xe;
                }
                M += me;
            }
            for (int d = 0; d < 3; ++d) {
                T->lo[3 * nd + d] = lo[d];
                T->hi[3 * nd + d] = hi[d];
                T->com[3 * nd + d] = M > 0.0 ? S[d] / M : 0.5 * ((double)lo[d] + (double)hi[d]);
            }
            T->mass[nd] = M;
        }
    }
}

static void orc_tree_free(orc_tree *T)
{
    free(T->lo);
    free(T->hi);
    free(T->mass);
    free(T->com);
}

/*
 * Short-range gravity of the active particles (NULL = all) on all n
 * (single periodic box of side L, r_cut <= L/4, theta <= 1). Outputs for
 * active i: acc (n x 3), scale = sum of |term| (the per-particle absolute
 * scale for tolerances), n_nodes / n_pairs = node and particle interactions.
 */
void orc_gravity(const uint32_t *X, int64_t n, double L, const double *m, double G, double theta,
                 double r_split, double r_cut, double h_soft, const int64_t *active, int64_t n_active,
                 double *acc, double *scale, int64_t *n_nodes, int64_t *n_pairs)
{
    uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * n);
    int64_t *sorted = (int64_t *)malloc(sizeof(int64_t) * n);
    orc_keys(X, n, 0, 0, key);
    orc_sort_keys(key, n, sorted);
    free(key);
    orc_tree T;
    orc_tree_build(X, m, sorted, n, &T);
    const double u = L / ORC_TWO32;           /* physical length of one integer unit */
    const double rcu = r_cut / L * 16777216.0; /* r_cut in coarse units (2^-24 L) */
    const uint64_t RCi = (uint64_t)ceil(rcu * rcu);
    const uint64_t P = (uint64_t)rint(theta * theta * 65536.0);
    int64_t na = active ? n_active : n;
#pragma omp parallel
    {
        int64_t *stack = (int64_t *)malloc(sizeof(int64_t) * 4096);
#pragma omp for schedule(dynamic, 16)
        for (int64_t a = 0; a < na; ++a) {
            int64_t i = active ? active[a] : a;
            const uint32_t *Xi = X + 3 * i;
            double ax = 0.0, ay = 0.0, az = 0.0, sc = 0.0;
            int64_t nn = 0, np = 0;
            /* stack entries: level * 2^40 + node index within the level */
            int sp = 0;
            stack[sp++] = (int64_t)(T.nlev - 1) << 40;
            while (sp > 0) {
                int64_t e = stack[--sp];
                int k = (int)(e >> 40);
                int64_t t = e & (((int64_t)1 << 40) - 1);
                if (k == 0) {
                    /* an opened leaf: its particles one by one */
                    int64_t p0 = 8 * t, p1 = p0 + 8 < n ? p0 + 8 : n;
                    for (int64_t p = p0; p < p1; ++p) {
                        int64_t j = sorted[p];
                        if (j == i) continue;
                        int32_t d[3];
                        uint64_t D2 = 0;
                        for (int q = 0; q < 3; ++q) {
                            d[q] = (int32_t)(X[3 * j + q] - Xi[q]);
                            uint64_t g = (uint64_t)(d[q] < 0 ? -(int64_t)d[q] : (int64_t)d[q]) >> 8;
                            D2 += g * g;
                        }
                        if (!(D2 < RCi)) continue;
                        ++np;
                        double rx = d[0] * u, ry = d[1] * u, rz = d[2] * u;
                        double r = sqrt(rx * rx + ry * ry + rz * rz);
                        if (r == 0.0) continue;
                        double f = G * m[j] * orc_grav_K(r, h_soft, r_split);
                        ax += f * rx;
                        ay += f * ry;
                        az += f * rz;
                        sc += fabs(f) * r;
                    }
                    continue;
                }
                /* an opened internal node: test its children */
                int64_t c0 = 8 * t, c1 = c0 + 8 < T.cnt[k - 1] ? c0 + 8 : T.cnt[k - 1];
                for (int64_t c = c0; c < c1; ++c) {
                    int64_t nd = T.off[k - 1] + c;
                    uint64_t D2 = 0, F2 = 0, l = 0;
                    for (int q = 0; q < 3; ++q) {
                        uint32_t lo = T.lo[3 * nd + q], hi = T.hi[3 * nd + q], x = Xi[q], gap = 0, far;
                        if (x < lo || x > hi) {
                            uint32_t g1 = lo - x, g2 = x - hi;   /* both ways round the periodic axis */
                            gap = g1 < g2 ? g1 : g2;
                            far = gap + (hi - lo);
                        } else {
                            far = x - lo > hi - x ? x - lo : hi - x;
                        }
                        uint64_t g = gap >> 8, f = ((uint64_t)far + 255) >> 8, s = (uint64_t)((hi - lo) >> 8);
                        D2 += g * g;
                        F2 += f * f;
                        if (s > l) l = s;
                    }
                    if (D2 >= RCi) continue;
                    uint64_t L2 = l * l;
                    if (P > 0 && D2 > 0 && F2 < RCi && L2 <= D2 && (L2 << 16) <= P * D2) {
                        ++nn;
                        double v[3];
                        for (int q = 0; q < 3; ++q) {
                            double dd = T.com[3 * nd + q] - (double)Xi[q];
                            dd -= ORC_TWO32 * rint(dd / ORC_TWO32);
                            v[q] = dd * u;
                        }
                        double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                        if (r == 0.0) continue;
                        double f = G * T.mass[nd] * orc_grav_K(r, h_soft, r_split);
                        ax += f * v[0];
                        ay += f * v[1];
                        az += f * v[2];
                        sc += fabs(f) * r;
                        continue;
                    }
                    stack[sp++] = ((int64_t)(k - 1) << 40) | c;
                }
            }
            acc[3 * i] = ax;
            acc[3 * i + 1] = ay;
            acc[3 * i + 2] = az;
            if (scale) scale[i] = sc;
            if (n_nodes) n_nodes[i] = nn;
            if (n_pairs) n_pairs[i] = np;
        }
        free(stack);
    }
    orc_tree_free(&T);
    free(sorted);
}
