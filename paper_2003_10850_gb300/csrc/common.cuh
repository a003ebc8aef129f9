// common.cuh -- shared device types and helpers of the GB300 SPH library.
//
// Geometry is exact integer geometry on the 2^32 lattice per axis: a
// particle's position is X = rint(frac(x/L) 2^32) mod 2^32 and the minimum-image
// separation is the two's-complement difference (int32)(X_j - X_i).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sph {

constexpr int kLeaf = 8;        // particles per leaf of the hierarchy
constexpr int kFan = 8;         // children per internal node
constexpr int kMaxLev = 12;     // levels per box (8 * 8^11 particles max)
constexpr int kWarp = 32;

// Device status bits (same values as SPH_ST_* in sph.h).
enum : uint32_t {
    ST_NOT_CONVERGED = 1u,
    ST_H_TOO_LARGE = 2u,
    ST_TIMEOUT = 4u,
    ST_INVALID = 8u,
};

// One periodic box of a grid. The hierarchy is implicit: level k node t of
// the box covers sorted particles [t*kLeaf*kFan^k, (t+1)*kLeaf*kFan^k) of the
// box; its children are level k-1 nodes [t*kFan, t*kFan + kFan). Only the
// bounding boxes (and h_max for the force pass) are stored, at global node
// index lvl_off[k] + t.
struct BoxDesc {
    long long off;          // first sorted particle of the box
    long long n;            // particles in the box
    double L;               // box side
    int nlev;               // number of levels; level nlev-1 is the single root
    int pow2;               // L is a power of two: h 2^32 / L = h S exactly
    int lvl_off[kMaxLev];   // global node index of the box's first node on level k
    int lvl_n[kMaxLev];     // nodes of the box on level k
    // FP32 forms for kernels that keep FP64 off their per-particle path
    float sf;               // L / 2^32 (box units per integer step), rounded to FP32
    float Lf;               // L rounded to FP32
    float wideL;            // 0.45 L: a leaf whose extent plus radius reaches it takes exact separations
    float capu;             // smallest float >= 0.5 L (1 - 1e-9), the bound h must stay below
    float Hs;               // 2^32 / L (integer steps per box unit), rounded to FP32
    double S;               // 2^32 / L in FP64 (correctly rounded; exact when pow2)
};

// Device counters and status of a context (cleared by sph_sync_status).
struct Counters {
    unsigned int status;
    unsigned int pad;
    unsigned long long density_pairs;
    unsigned long long force_pairs;
    unsigned long long density_evals;
    unsigned long long pair_tests;
    unsigned long long groups;
    unsigned long long grav_nodes;
    unsigned long long grav_pairs;
    unsigned long long list_force;
};

// -------------------------------------------------------------------------
// Small helpers
// -------------------------------------------------------------------------

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Periodic gap (integer units, >= 0) between the closed intervals [a0,a1] and
// [b0,b1] on the circle of circumference 2^32: the minimum over the three
// images b, b+2^32, b-2^32 of the ordinary interval gap.
__device__ __forceinline__ float periodic_gap(uint32_t a0, uint32_t a1, uint32_t b0, uint32_t b1) {
    const long long two32 = 1ll << 32;
    long long d1 = (long long)b0 - (long long)a1;  // b to the right of a
    long long d2 = (long long)a0 - (long long)b1;  // b to the left of a
    long long g = max(0ll, max(d1, d2));
    g = min(g, d1 + two32);
    g = min(g, d2 + two32);
    return (float)g;
}

// splitmix64 finaliser (Steele, Lea, Flood 2014) for neighbour-set checksums.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// -------------------------------------------------------------------------
// Kernel function: M4 cubic spline with support h, branch-free form.
//   w(q)  = 2 a^3 - 8 b^3,   a = max(1-q,0), b = max(1/2-q,0)
//   w'(q) = -6 a^2 + 24 b^2
// which equals 1 - 6q^2 + 6q^3 on [0,1/2], 2(1-q)^3 on [1/2,1], 0 beyond.
// -------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void spline(T q, T& w, T& dw) {
    T a = max(T(1) - q, T(0));
    T b = max(T(0.5) - q, T(0));
    T a2 = a * a, b2 = b * b;
    w = T(2) * a2 * a - T(8) * b2 * b;
    dw = T(24) * b2 - T(6) * a2;
}

// Compensated (Kahan) addition of x into (s, c); explicit round-to-nearest
// intrinsics keep the compensation from being reassociated or contracted.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
    float y = __fsub_rn(x, c);
    float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}
__device__ __forceinline__ void kahan_add(double& s, double& c, double x) {
    double y = __dsub_rn(x, c);
    double t = __dadd_rn(s, y);
    c = __dsub_rn(__dsub_rn(t, s), y);
    s = t;
}

// Exact neighbour predicate: (double)D2 < HH with D2 the exact integer
// squared distance and HH = (h 2^32 / L)^2 in FP64 -- the single IEEE
// rounding of D2 and the FP64 product are what the definition prescribes.
__device__ __forceinline__ unsigned long long exact_d2(uint4 a, uint4 b) {
    long long dx = (int)(a.x - b.x), dy = (int)(a.y - b.y), dz = (int)(a.z - b.z);
    return (unsigned long long)(dx * dx) + (unsigned long long)(dy * dy) +
           (unsigned long long)(dz * dz);
}
__device__ __forceinline__ bool exact_pred(unsigned long long D2, double HH) {
    return __ull2double_rn(D2) < HH;
}

}  // namespace sph
