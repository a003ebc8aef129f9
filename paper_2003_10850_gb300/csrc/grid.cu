// grid.cu -- quantisation, Morton keys, LSD radix sort, and the implicit
// bounding-volume hierarchy over Morton-sorted particles.
//
// The paper's modules each walk a tree to find the neighbours of active
// particles (Sec. 1, Sec. 2.4); its tree is built on the CPU, which it names
// as a coming bottleneck (Sec. 4). Here the whole neighbour structure is built
// on the GPU: integer positions -> 63-bit Morton keys -> stable radix sort ->
// fixed fan-out hierarchy whose level-k node t covers sorted particles
// [t*8^(k+1), (t+1)*8^(k+1)) of its box, with integer bounding boxes.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "internal.cuh"

namespace sph {

// ---------------------------------------------------------------------------
// a1: quantise + key
// ---------------------------------------------------------------------------

// Spread the low 21 bits of v so that bit b lands at bit 3b (bit tricks of
// the usual "part1by2" form on 64-bit words).
__device__ __forceinline__ unsigned long long spread3(unsigned v) {
    unsigned long long x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// x / L is a product when L is a power of two: x * (S 2^-32) with S = 2^32 / L
// exact, so the value is the division's (FP64 division is a long sequence on
// the narrow FP64 pipe).
__device__ __forceinline__ unsigned quantize1(double x, const BoxDesc& B, bool& bad) {
    if (!isfinite(x)) { bad = true; return 0u; }
    double t = B.pow2 ? x * (B.S * 2.3283064365386962890625e-10) : x / B.L;
    t = t - floor(t);
    double v = rint(t * 4294967296.0);
    if (v >= 4294967296.0) v -= 4294967296.0;
    return (unsigned)(unsigned long long)v;
}

// FP32 positions inside [0, L) of a power-of-two box take an FP32 path with
// the same result: t = x / L is in [0, 1), so frac(t) = t, and t 2^32 = x Hs
// (Hs = 2^32 / L, a power of two) is exact in FP32; rint of that float is the
// FP64 rint of the same value. Everything else takes the FP64 definition.
__device__ __forceinline__ unsigned quantize_p(float x, const BoxDesc& B, bool& bad) {
    if (B.pow2 && x >= 0.f && x < B.Lf && (double)B.Lf == B.L) {
        const float v = rintf(x * B.Hs);
        return v >= 4294967296.0f ? 0u : (unsigned)(unsigned long long)v;
    }
    return quantize1((double)x, B, bad);
}
__device__ __forceinline__ unsigned quantize_p(double x, const BoxDesc& B, bool& bad) {
    return quantize1(x, B, bad);
}

template <typename P>
__global__ void k_quantize(const P* __restrict__ pos, const float* __restrict__ mass, int n,
                           const long long* __restrict__ box_off, const BoxDesc* __restrict__ boxes,
                           int nb, int bb, uint4* __restrict__ xq, unsigned long long* __restrict__ keys,
                           unsigned* __restrict__ vals, Counters* ctr) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = nb - 1;  // largest b with box_off[b] <= i
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (box_off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    const BoxDesc& B = boxes[lo];
    bool bad = false;
    unsigned X = quantize_p(pos[3 * (size_t)i], B, bad);
    unsigned Y = quantize_p(pos[3 * (size_t)i + 1], B, bad);
    unsigned Z = quantize_p(pos[3 * (size_t)i + 2], B, bad);
    float m = mass[i];
    if (!(m > 0.f) || !isfinite(m)) bad = true;
    if (bad) atomicOr(&ctr->status, ST_INVALID);
    unsigned long long key = (spread3(X >> 11) << 2) | (spread3(Y >> 11) << 1) | spread3(Z >> 11);
    if (bb) key = ((unsigned long long)lo << (63 - bb)) | (key >> bb);
    xq[i] = make_uint4(X, Y, Z, __float_as_uint(m));
    keys[i] = key;
    vals[i] = (unsigned)i;
}

// ---------------------------------------------------------------------------
// Exclusive scan (reduce, scan the block sums, apply), 4096 items per block
// ---------------------------------------------------------------------------

constexpr int kScanT = 1024, kScanIPT = 4, kScanTile = kScanT * kScanIPT;

__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned* sm, unsigned& total) {
    // sm: 32 words. Returns the exclusive prefix of v over the block.
    unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    if (lane == 31) sm[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned nw = blockDim.x >> 5;
        unsigned w = lane < nw ? sm[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= (unsigned)o) w += y;
        }
        sm[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    total = sm[(blockDim.x >> 5) - 1];
    unsigned before = warp ? sm[warp - 1] : 0u;
    unsigned r = before + x - v;
    __syncthreads();
    return r;
}

template <typename In>
__global__ void k_scan_reduce(const In* __restrict__ in, int n, unsigned* __restrict__ bsum) {
    __shared__ unsigned sm[32];
    int base = blockIdx.x * kScanTile + threadIdx.x * kScanIPT;
    unsigned s = 0;
#pragma unroll
    for (int k = 0; k < kScanIPT; ++k)
        if (base + k < n) s += (unsigned)in[base + k];
    unsigned tot;
    block_excl_scan(s, sm, tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_bsums(unsigned* bsum, int nb) {
    __shared__ unsigned sm[32];
    unsigned carry = 0;
    for (int base = 0; base < nb; base += blockDim.x) {
        int i = base + threadIdx.x;
        unsigned v = i < nb ? bsum[i] : 0u;
        unsigned tot;
        unsigned ex = block_excl_scan(v, sm, tot);
        if (i < nb) bsum[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) bsum[nb] = carry;
}

template <typename In>
__global__ void k_scan_apply(const In* __restrict__ in, int n, const unsigned* __restrict__ bsum,
                             unsigned* __restrict__ out) {
    __shared__ unsigned sm[32];
    int base = blockIdx.x * kScanTile + threadIdx.x * kScanIPT;
    unsigned v[kScanIPT], s = 0;
#pragma unroll
    for (int k = 0; k < kScanIPT; ++k) {
        v[k] = (base + k < n) ? (unsigned)in[base + k] : 0u;
        s += v[k];
    }
    unsigned tot;
    unsigned ex = block_excl_scan(s, sm, tot) + bsum[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanIPT; ++k) {
        if (base + k < n) out[base + k] = ex;
        ex += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = bsum[gridDim.x];
}

template <typename In>
void scan_exclusive(const In* in, int n, uint32_t* out, uint32_t* tmp, cudaStream_t s, unsigned* nl) {
    int nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 0) {
        cudaMemsetAsync(out, 0, sizeof(uint32_t), s);
        return;
    }
    k_scan_reduce<In><<<nb, kScanT, 0, s>>>(in, n, tmp);
    k_scan_bsums<<<1, 1024, 0, s>>>(tmp, nb);
    k_scan_apply<In><<<nb, kScanT, 0, s>>>(in, n, tmp, out);
    *nl += 3;
}
template void scan_exclusive<uint8_t>(const uint8_t*, int, uint32_t*, uint32_t*, cudaStream_t, unsigned*);
template void scan_exclusive<uint32_t>(const uint32_t*, int, uint32_t*, uint32_t*, cudaStream_t, unsigned*);

// ---------------------------------------------------------------------------
// a2: stable LSD radix sort of (64-bit key, 32-bit value), 8-bit digits
// ---------------------------------------------------------------------------

constexpr int kRsT = 256, kRsIPT = 16, kRsTile = kRsT * kRsIPT;

__global__ void k_rs_hist(const unsigned long long* __restrict__ keys, int n, int shift,
                          unsigned* __restrict__ counts, int nblk) {
    __shared__ unsigned hist[256];
    hist[threadIdx.x] = 0;
    __syncthreads();
    int base = blockIdx.x * kRsTile;
#pragma unroll 4
    for (int r = 0; r < kRsIPT; ++r) {
        int k = base + r * kRsT + threadIdx.x;
        if (k < n) atomicAdd(&hist[(unsigned)(keys[k] >> shift) & 255u], 1u);
    }
    __syncthreads();
    counts[threadIdx.x * nblk + blockIdx.x] = hist[threadIdx.x];
}

// Each block ranks its tile in rounds of 256 consecutive items; within a
// round the rank of an item among equal digits is (items of earlier warps) +
// (earlier lanes of its warp with the same digit), so the order of equal
// digits is preserved (stable). The ranks place the tile's items in digit
// order in shared memory (their tile indices); the items are then written
// out in that order, so that consecutive threads write consecutive places of
// a digit's run (coalesced) instead of one scattered place each.
__global__ void __launch_bounds__(kRsT) k_rs_scatter(const unsigned long long* __restrict__ kin,
                                                     const unsigned* __restrict__ vin,
                                                     unsigned long long* __restrict__ kout,
                                                     unsigned* __restrict__ vout, int n, int shift,
                                                     const unsigned* __restrict__ offs,
                                                     const unsigned* __restrict__ counts, int nblk) {
    __shared__ unsigned short at[kRsTile];     // tile index of the item at each place of the tile
    __shared__ unsigned start[256];             // first place of each digit's run in the tile
    __shared__ unsigned run[256];               // places taken so far by each digit
    __shared__ unsigned wcnt[kRsT / 32][256];
    __shared__ unsigned wsum[kRsT / 32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // exclusive scan of the tile's digit counts (one digit per thread)
    {
        const unsigned c = counts[tid * nblk + blockIdx.x];
        unsigned x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        unsigned w0 = 0;
        for (int w = 0; w < warp; ++w) w0 += wsum[w];
        start[tid] = w0 + x - c;
        run[tid] = w0 + x - c;
    }
#pragma unroll
    for (int w = 0; w < kRsT / 32; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    const int tile = blockIdx.x * kRsTile;
    for (int r = 0; r < kRsIPT; ++r) {
        const int k = tile + r * kRsT + tid;
        const bool valid = k < n;
        const unsigned d = valid ? ((unsigned)(kin[k] >> shift) & 255u) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const unsigned lt = peers & ((1u << lane) - 1u);
        if (valid && lt == 0u) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        {
            unsigned s = run[tid];
#pragma unroll
            for (int w = 0; w < kRsT / 32; ++w) {
                const unsigned t = wcnt[w][tid];
                wcnt[w][tid] = s;
                s += t;
            }
            run[tid] = s;
        }
        __syncthreads();
        if (valid) at[wcnt[warp][d] + __popc(lt)] = (unsigned short)(r * kRsT + tid);
        __syncthreads();
#pragma unroll
        for (int w = 0; w < kRsT / 32; ++w) wcnt[w][tid] = 0;
        __syncthreads();
    }
    // write out in place order: place p of digit d goes to its run's global start
    const int tn = min(kRsTile, n - tile);
    for (int p = tid; p < tn; p += kRsT) {
        const int i = tile + (int)at[p];
        const unsigned long long key = kin[i];
        const unsigned d = (unsigned)(key >> shift) & 255u;
        const unsigned g = offs[d * nblk + blockIdx.x] + ((unsigned)p - start[d]);
        kout[g] = key;
        vout[g] = vin[i];
    }
}

static void radix_sort(unsigned long long* keys, unsigned* vals, unsigned long long* keys2,
                       unsigned* vals2, int n, int end_bit, unsigned* counts, unsigned* cscan,
                       unsigned* tmp, cudaStream_t s, unsigned* nl) {
    int nblk = (n + kRsTile - 1) / kRsTile;
    unsigned long long *ka = keys, *kb = keys2;
    unsigned *va = vals, *vb = vals2;
    for (int shift = 0; shift < end_bit; shift += 8) {
        k_rs_hist<<<nblk, kRsT, 0, s>>>(ka, n, shift, counts, nblk);
        scan_exclusive<uint32_t>(counts, 256 * nblk, cscan, tmp, s, nl);
        k_rs_scatter<<<nblk, kRsT, 0, s>>>(ka, va, kb, vb, n, shift, cscan, counts, nblk);
        *nl += 2;
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        cudaMemcpyAsync(keys, ka, sizeof(unsigned long long) * n, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(vals, va, sizeof(unsigned) * n, cudaMemcpyDeviceToDevice, s);
    }
}

// ---------------------------------------------------------------------------
// a3: gather into sorted order, hierarchy bounding boxes, h_max
// ---------------------------------------------------------------------------

__global__ void k_gather(const uint4* __restrict__ xq, const unsigned* __restrict__ sorted_vals, int n,
                         uint4* __restrict__ posm, int32_t* __restrict__ perm, int32_t* __restrict__ rank) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int i = (int)sorted_vals[k];
    posm[k] = xq[i];
    perm[k] = i;
    rank[i] = k;
}

// Node centre (integer) and half extents (box units, padded by two integer
// units) -- the form the thread-per-particle walk tests against.
__device__ __forceinline__ void node_geom(uint4 a, uint4 b, double s, uint4& c, float4& e) {
    c = make_uint4(a.x + ((b.x - a.x) >> 1), a.y + ((b.y - a.y) >> 1), a.z + ((b.z - a.z) >> 1), 0u);
    e = make_float4((float)((double)(((b.x - a.x) >> 1) + 2u) * s), (float)((double)(((b.y - a.y) >> 1) + 2u) * s),
                    (float)((double)(((b.z - a.z) >> 1) + 2u) * s), 0.f);
}

__global__ void k_leaf_bbox(const uint4* __restrict__ posm, const BoxDesc* __restrict__ boxes,
                            uint4* __restrict__ lo, uint4* __restrict__ hi, uint4* __restrict__ nc,
                            float4* __restrict__ ne, float4* __restrict__ posf) {
    const BoxDesc& B = boxes[blockIdx.y];
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B.lvl_n[0]) return;
    long long p0 = B.off + (long long)t * kLeaf, p1 = min(p0 + kLeaf, B.off + B.n);
    uint4 a = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0), b = make_uint4(0, 0, 0, 0);
    for (long long p = p0; p < p1; ++p) {
        uint4 x = posm[p];
        a.x = min(a.x, x.x); a.y = min(a.y, x.y); a.z = min(a.z, x.z);
        b.x = max(b.x, x.x); b.y = max(b.y, x.y); b.z = max(b.z, x.z);
    }
    const int nd = B.lvl_off[0] + t;
    lo[nd] = a;
    hi[nd] = b;
    const double s = ldexp(B.L, -32);
    uint4 c;
    float4 e;
    node_geom(a, b, s, c, e);
    nc[nd] = c;
    ne[nd] = e;
    // leaf-relative FP32 coordinates (box units) and mass of the leaf's particles
    const float sf = (float)s;
    for (long long p = p0; p < p1; ++p) {
        uint4 x = posm[p];
        posf[p] = make_float4((float)(int)(x.x - c.x) * sf, (float)(int)(x.y - c.y) * sf,
                              (float)(int)(x.z - c.z) * sf, __uint_as_float(x.w));
    }
}

__global__ void k_node_bbox(int lev, const BoxDesc* __restrict__ boxes, uint4* __restrict__ lo,
                            uint4* __restrict__ hi, uint4* __restrict__ nc, float4* __restrict__ ne) {
    const BoxDesc& B = boxes[blockIdx.y];
    if (lev >= B.nlev) return;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B.lvl_n[lev]) return;
    int c0 = t * kFan, c1 = min(c0 + kFan, B.lvl_n[lev - 1]);
    uint4 a = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0), b = make_uint4(0, 0, 0, 0);
    for (int c = c0; c < c1; ++c) {
        uint4 x = lo[B.lvl_off[lev - 1] + c], y = hi[B.lvl_off[lev - 1] + c];
        a.x = min(a.x, x.x); a.y = min(a.y, x.y); a.z = min(a.z, x.z);
        b.x = max(b.x, y.x); b.y = max(b.y, y.y); b.z = max(b.z, y.z);
    }
    const int nd = B.lvl_off[lev] + t;
    lo[nd] = a;
    hi[nd] = b;
    uint4 c;
    float4 e;
    node_geom(a, b, ldexp(B.L, -32), c, e);
    nc[nd] = c;
    ne[nd] = e;
}

__global__ void k_leaf_hmax(const int32_t* __restrict__ perm, const float* __restrict__ h,
                            const BoxDesc* __restrict__ boxes, float* __restrict__ hmax, float4* __restrict__ ne) {
    const BoxDesc& B = boxes[blockIdx.y];
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B.lvl_n[0]) return;
    long long p0 = B.off + (long long)t * kLeaf, p1 = min(p0 + kLeaf, B.off + B.n);
    float m = 0.f;
    for (long long p = p0; p < p1; ++p) m = fmaxf(m, h[perm[p]]);
    hmax[B.lvl_off[0] + t] = m;
    ne[B.lvl_off[0] + t].w = m;
}

__global__ void k_node_hmax(int lev, const BoxDesc* __restrict__ boxes, float* __restrict__ hmax,
                            float4* __restrict__ ne) {
    const BoxDesc& B = boxes[blockIdx.y];
    if (lev >= B.nlev) return;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B.lvl_n[lev]) return;
    int c0 = t * kFan, c1 = min(c0 + kFan, B.lvl_n[lev - 1]);
    float m = 0.f;
    for (int c = c0; c < c1; ++c) m = fmaxf(m, hmax[B.lvl_off[lev - 1] + c]);
    hmax[B.lvl_off[lev] + t] = m;
    ne[B.lvl_off[lev] + t].w = m;
}

// ---------------------------------------------------------------------------
// a6: active list
// ---------------------------------------------------------------------------

__global__ void k_iota(int32_t* a, int n) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) a[k] = k;
}

// all particles active: the identity list, and its length where the subset
// path leaves the compacted count (scan[n])
__global__ void k_iota_count(int32_t* a, int n, uint32_t* count) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) a[k] = k;
    if (k == 0) *count = (uint32_t)n;
}

__global__ void k_mark(const int32_t* __restrict__ active, int na, const int32_t* __restrict__ rank,
                       uint8_t* __restrict__ flag, int n, Counters* ctr) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= na) return;
    int i = active[k];
    if (i < 0) return;   // a padding entry (a list of fixed capacity whose count lives on the device)
    if (i >= n) { atomicOr(&ctr->status, ST_INVALID); return; }
    flag[rank[i]] = 1;
}

__global__ void k_compact(const uint8_t* __restrict__ flag, const uint32_t* __restrict__ scan, int n,
                          int32_t* __restrict__ act) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n && flag[k]) act[scan[k]] = k;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

#define GRID_CHECK(call)                                                                  \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            ctx->err = std::string("CUDA error in grid build: ") + cudaGetErrorString(e_); \
            grid_free(g);                                                                 \
            return e_ == cudaErrorMemoryAllocation ? SPH_ERR_OOM : SPH_ERR_CUDA;          \
        }                                                                                 \
    } while (0)

void grid_free(sph_grid* g) {
    if (!g) return;
    void* ptrs[] = {g->boxes, g->posm, g->xq, g->perm, g->rank, g->keys, g->node_lo, g->node_hi,
                    g->node_hmax, g->act, g->flag, g->scan, g->scan_tmp, g->list_a, g->list_b, g->st_lo, g->st_hi, g->list_n, g->d_off, g->d_L,
                    g->k2, g->v1, g->v2, g->counts, g->cscan, g->node_c, g->node_e, g->posf,
                    g->fvel, g->fthermo, g->fposh, g->fvm, g->fbal, g->fcond, g->fvisc, g->node_m, g->box_rci, g->nbr, g->nbr_off, g->nbr_n, g->ext_n, g->ext, g->list_xh, g->list_st, g->fb_list, g->list_ep, g->mp_x, g->bw_ga, g->bw_xbar, g->bw_rd, g->bw_f, g->mp_j, g->den_left};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete g;
}

static void grid_fill(sph_grid* g, const void* pos, int f64, const float* mass, cudaStream_t s) {
    sph_ctx* ctx = g->ctx;
    const int n = (int)g->n, nb = g->n_boxes;
    const int blocks = (n + 255) / 256;
    if (f64)
        k_quantize<double><<<blocks, 256, 0, s>>>((const double*)pos, mass, n, g->d_off, g->boxes, nb, g->box_bits,
                                                  g->xq, (unsigned long long*)g->keys, g->v1, ctx->counters);
    else
        k_quantize<float><<<blocks, 256, 0, s>>>((const float*)pos, mass, n, g->d_off, g->boxes, nb, g->box_bits,
                                                 g->xq, (unsigned long long*)g->keys, g->v1, ctx->counters);
    ++ctx->launches;
    radix_sort((unsigned long long*)g->keys, g->v1, g->k2, g->v2, n, 63, g->counts, g->cscan, g->scan_tmp, s,
               &ctx->launches);
    k_gather<<<blocks, 256, 0, s>>>(g->xq, g->v1, n, g->posm, g->perm, g->rank);
    dim3 lg((g->max_leaves + 127) / 128, nb);
    k_leaf_bbox<<<lg, 128, 0, s>>>(g->posm, g->boxes, g->node_lo, g->node_hi, g->node_c, g->node_e, g->posf);
    ctx->launches += 2;
    for (int lev = 1; lev < g->max_lev; ++lev) {
        dim3 ng((g->lvl_max[lev] + 127) / 128, nb);
        k_node_bbox<<<ng, 128, 0, s>>>(lev, g->boxes, g->node_lo, g->node_hi, g->node_c, g->node_e);
        ++ctx->launches;
    }
}

sph_status grid_build(sph_ctx* ctx, const void* pos, int f64, const float* mass, bool lists, const int64_t* offs,
                      const double* Ls, int nb, cudaStream_t s, sph_grid** out) {
    sph_grid* g = new sph_grid();
    g->ctx = ctx;
    g->device = ctx->device;
    const int n = (int)offs[nb];
    g->n = n;
    g->n_boxes = nb;
    int bb = 0;
    while ((1 << bb) < nb) ++bb;
    g->box_bits = bb;
    // implicit hierarchy layout, box-major, level-minor
    g->boxes_h.resize(nb);
    int node = 0, maxleaf = 0, maxlev = 0;
    for (int b = 0; b < nb; ++b) {
        BoxDesc& B = g->boxes_h[b];
        B = BoxDesc();
        B.off = offs[b];
        B.n = offs[b + 1] - offs[b];
        B.L = Ls[b];
        int cnt = (int)((B.n + kLeaf - 1) / kLeaf), lev = 0;
        while (true) {
            if (lev >= kMaxLev) { ctx->err = "box too large for the hierarchy"; delete g; return SPH_ERR_INVALID; }
            B.lvl_off[lev] = node;
            B.lvl_n[lev] = cnt;
            g->lvl_max[lev] = std::max(g->lvl_max[lev], cnt);
            node += cnt;
            ++lev;
            if (cnt == 1) break;
            cnt = (cnt + kFan - 1) / kFan;
        }
        B.nlev = lev;
        B.sf = (float)std::ldexp(B.L, -32);
        B.S = 4294967296.0 / B.L;
        B.Hs = (float)B.S;
        int ex = 0;
        B.pow2 = std::frexp(B.L, &ex) == 0.5 ? 1 : 0;
        B.Lf = (float)B.L;
        B.wideL = 0.45f * B.Lf;
        const double cap = 0.5 * B.L * (1.0 - 1e-9);
        B.capu = (float)cap;
        if ((double)B.capu < cap) B.capu = std::nextafter(B.capu, INFINITY);
        maxlev = std::max(maxlev, lev);
        maxleaf = std::max(maxleaf, B.lvl_n[0]);
    }
    g->n_nodes = node;
    g->max_leaves = maxleaf;
    g->max_lev = maxlev;

    const int nblk = (n + kRsTile - 1) / kRsTile;
    const int scan_words = 256 * nblk + 1;
    const int tmp_words = std::max(n, scan_words) / kScanTile + 4;
    GRID_CHECK(cudaMalloc(&g->boxes, sizeof(BoxDesc) * nb));
    GRID_CHECK(cudaMemcpyAsync(g->boxes, g->boxes_h.data(), sizeof(BoxDesc) * nb, cudaMemcpyHostToDevice, s));
    GRID_CHECK(cudaMalloc(&g->d_off, sizeof(long long) * (nb + 1)));
    GRID_CHECK(cudaMalloc(&g->d_L, sizeof(double) * nb));
    {
        std::vector<long long> offh(offs, offs + nb + 1);
        GRID_CHECK(cudaMemcpyAsync(g->d_off, offh.data(), sizeof(long long) * (nb + 1), cudaMemcpyHostToDevice, s));
        GRID_CHECK(cudaMemcpyAsync(g->d_L, Ls, sizeof(double) * nb, cudaMemcpyHostToDevice, s));
        GRID_CHECK(cudaStreamSynchronize(s));  // host staging buffers go out of scope
    }
    GRID_CHECK(cudaMalloc(&g->posm, sizeof(uint4) * n));
    GRID_CHECK(cudaMalloc(&g->xq, sizeof(uint4) * n));
    GRID_CHECK(cudaMalloc(&g->perm, sizeof(int32_t) * n));
    GRID_CHECK(cudaMalloc(&g->rank, sizeof(int32_t) * n));
    GRID_CHECK(cudaMalloc(&g->keys, sizeof(uint64_t) * n));
    GRID_CHECK(cudaMalloc(&g->node_lo, sizeof(uint4) * node));
    GRID_CHECK(cudaMalloc(&g->node_hi, sizeof(uint4) * node));
    GRID_CHECK(cudaMalloc(&g->node_hmax, sizeof(float) * node));
    GRID_CHECK(cudaMalloc(&g->node_c, sizeof(uint4) * node));
    GRID_CHECK(cudaMalloc(&g->node_e, sizeof(float4) * node));
    GRID_CHECK(cudaMemset(g->node_e, 0, sizeof(float4) * node));
    GRID_CHECK(cudaMalloc(&g->posf, sizeof(float4) * n));
    GRID_CHECK(cudaMalloc(&g->fvel, sizeof(float4) * n));
    GRID_CHECK(cudaMalloc(&g->fthermo, sizeof(float4) * n));
    GRID_CHECK(cudaMalloc(&g->fposh, sizeof(float4) * n));
    GRID_CHECK(cudaMalloc(&g->fvm, sizeof(float4) * n));
    GRID_CHECK(cudaMalloc(&g->fbal, sizeof(float) * n));
    GRID_CHECK(cudaMalloc(&g->fcond, sizeof(float2) * n));
    GRID_CHECK(cudaMalloc(&g->fvisc, sizeof(float2) * n));
    GRID_CHECK(cudaMalloc(&g->node_m, sizeof(float4) * node));
    GRID_CHECK(cudaMalloc(&g->box_rci, sizeof(unsigned long long) * nb));
    // the near-list indices of the density pass's member-parallel path, one
    // block of kMpMembers x kMpCap per persistent warp
    GRID_CHECK(cudaMalloc(&g->mp_j, sizeof(int32_t) * (size_t)ctx->sm_count * kMpWarpsPerSm * kMpMembers * kMpCap));
    GRID_CHECK(cudaMalloc(&g->den_left, sizeof(int32_t) * n));
    if (lists) {
        // Neighbour-list pools (int32 offsets: at most 2^31 - 2^12 entries each).
        // Lists are an optimisation: if they cannot be allocated the grid is
        // built without them and the force pass walks.
        const long long lim = (1ll << 31) - (1ll << 12);
        g->list_pool = (int64_t)std::min<long long>((long long)n * kListPool, lim);
        void** lp[] = {(void**)&g->nbr, (void**)&g->nbr_off, (void**)&g->nbr_n, (void**)&g->ext_n,
                       (void**)&g->ext, (void**)&g->list_xh, (void**)&g->list_st, (void**)&g->fb_list,
                       (void**)&g->list_ep, (void**)&g->mp_x};
        const size_t sz[] = {sizeof(int32_t) * (size_t)g->list_pool, sizeof(int32_t) * n, sizeof(int32_t) * n,
                             sizeof(uint32_t) * n, sizeof(int32_t) * (size_t)n * kExtCap, sizeof(uint4) * n,
                             sizeof(unsigned) * kListSt, sizeof(int32_t) * n, sizeof(uint32_t) * n,
                             sizeof(int32_t) * (size_t)ctx->sm_count * kMpWarpsPerSm * kMpMembers * kMpFar};
        bool ok = true;
        for (int k = 0; k < 10 && ok; ++k) ok = cudaMalloc(lp[k], sz[k]) == cudaSuccess;
        if (ok) ok = cudaMemset(g->list_st, 0, sizeof(unsigned) * kListSt) == cudaSuccess;
        if (ok) ok = cudaMemset(g->list_ep, 0, sizeof(uint32_t) * n) == cudaSuccess;
        if (!ok) {
            (void)cudaGetLastError();
            for (void** q : lp) {
                if (*q) cudaFree(*q);
                *q = nullptr;
            }
        }
    }
    GRID_CHECK(cudaMalloc(&g->act, sizeof(int32_t) * n));
    GRID_CHECK(cudaMalloc(&g->flag, n));
    GRID_CHECK(cudaMalloc(&g->scan, sizeof(uint32_t) * (n + 1)));
    GRID_CHECK(cudaMalloc(&g->scan_tmp, sizeof(uint32_t) * tmp_words));
    GRID_CHECK(cudaMalloc(&g->list_a, sizeof(int32_t) * n));
    GRID_CHECK(cudaMalloc(&g->list_b, sizeof(int32_t) * n));
    GRID_CHECK(cudaMalloc(&g->st_lo, sizeof(float) * n));
    GRID_CHECK(cudaMalloc(&g->st_hi, sizeof(float) * n));
    GRID_CHECK(cudaMalloc(&g->list_n, sizeof(int) * 2));
    GRID_CHECK(cudaMalloc(&g->k2, sizeof(unsigned long long) * n));
    GRID_CHECK(cudaMalloc(&g->v1, sizeof(unsigned) * n));
    GRID_CHECK(cudaMalloc(&g->v2, sizeof(unsigned) * n));
    GRID_CHECK(cudaMalloc(&g->counts, sizeof(unsigned) * scan_words));
    GRID_CHECK(cudaMalloc(&g->cscan, sizeof(unsigned) * (scan_words + 1)));
    grid_fill(g, pos, f64, mass, s);
    GRID_CHECK(cudaGetLastError());
    GRID_CHECK(cudaStreamSynchronize(s));
    *out = g;
    return SPH_OK;
}

sph_status grid_update(sph_grid* g, const void* pos, int f64, const float* mass, cudaStream_t s) {
    g->lists_rec = false;   // the particles may have moved: recorded neighbour lists are stale
    grid_fill(g, pos, f64, mass, s);
    cudaError_t e = cudaGetLastError();
    if (e) {
        g->ctx->err = std::string("CUDA error in grid update: ") + cudaGetErrorString(e);
        return SPH_ERR_CUDA;
    }
    return SPH_OK;
}

void grid_refresh_hmax(sph_grid* g, const float* h, cudaStream_t s) {
    int nb = g->n_boxes;
    dim3 lg((g->max_leaves + 127) / 128, nb);
    k_leaf_hmax<<<lg, 128, 0, s>>>(g->perm, h, g->boxes, g->node_hmax, g->node_e);
    ++g->ctx->launches;
    for (int lev = 1; lev < g->max_lev; ++lev) {
        dim3 ng((g->lvl_max[lev] + 127) / 128, nb);
        k_node_hmax<<<ng, 128, 0, s>>>(lev, g->boxes, g->node_hmax, g->node_e);
        ++g->ctx->launches;
    }
}

void grid_active(sph_grid* g, const int32_t* active, int64_t n_active, cudaStream_t s) {
    int n = (int)g->n;
    unsigned& nl = g->ctx->launches;
    if (!active) {
        k_iota_count<<<(n + 255) / 256, 256, 0, s>>>(g->act, n, g->scan + n);
        ++nl;
    } else {
        cudaMemsetAsync(g->flag, 0, n, s);
        if (n_active > 0) {
            k_mark<<<(int)((n_active + 255) / 256), 256, 0, s>>>(active, (int)n_active, g->rank, g->flag, n,
                                                                  g->ctx->counters);
            ++nl;
        }
        scan_exclusive<uint8_t>(g->flag, n, g->scan, g->scan_tmp, s, &nl);
        k_compact<<<(n + 255) / 256, 256, 0, s>>>(g->flag, g->scan, n, g->act);
        ++nl;
    }
}

}  // namespace sph
