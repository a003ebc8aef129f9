// noalloc.cu -- sph_sort_keys_static: the stable (key, index) radix sort of
// the grid build, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or budget (where every device byte is accounted
// for), code on a time-critical loop where cudaMalloc's implicit device
// synchronisation is not acceptable, or callers without a sph_ctx (creating
// one allocates). This entry point allocates nothing: its scratch -- the
// second key/index buffer and the digit histograms of the radix passes -- is
// the file-scope device array below, of a fixed size, which every GPU that
// loads the library holds until the process exits.
#include "internal.cuh"

namespace sph {
// kernels of the grid build (grid.cu), reused unchanged
__global__ void k_rs_hist(const unsigned long long* keys, int n, int shift, unsigned* counts, int nblk);
__global__ void k_rs_scatter(const unsigned long long* kin, const unsigned* vin, unsigned long long* kout,
                             unsigned* vout, int n, int shift, const unsigned* offs, const unsigned* counts,
                             int nblk);
__global__ void k_iota(int32_t* a, int n);
}  // namespace sph

namespace {

constexpr int kMaxKeys = SPH_SORT_STATIC_MAX_KEYS;
constexpr int kTile = 4096;                            // keys per block of a radix pass
constexpr int kBlocks = (kMaxKeys + kTile - 1) / kTile;
constexpr int kCountWords = 256 * kBlocks + 1;

// byte offsets of the sub-buffers (each 256-byte aligned)
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffKeys = 0;
constexpr size_t kOffVals = align256(kOffKeys + sizeof(unsigned long long) * kMaxKeys);
constexpr size_t kOffCounts = align256(kOffVals + sizeof(unsigned) * kMaxKeys);
constexpr size_t kOffScan = align256(kOffCounts + sizeof(unsigned) * kCountWords);
constexpr size_t kOffTmp = align256(kOffScan + sizeof(unsigned) * (kCountWords + 1));
constexpr size_t kScratchBytes = align256(kOffTmp + sizeof(unsigned) * 64);

// The scratch itself. Host code must not use this name as a device address:
// on the host it names a stand-in object; the device address comes from
// cudaGetSymbolAddress below. Device code could name it directly; the radix
// kernels are shared with the grid build and take plain pointers instead.
static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

// The array's device address in the current device's context. Looked up on
// every call (cudaGetSymbolAddress allocates nothing), so a context that was
// destroyed and created again (cudaDeviceReset) never leaves a stale address
// behind. Under lazy module loading (CUDA_MODULE_LOADING=LAZY, the default) the
// first lookup on a device loads this module, which creates the array: that
// first call is the set-up, and it should come before any stream capture and
// outside any memory budget.
sph_status scratch_for_current_device(unsigned char** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) return SPH_ERR_CUDA;
    *out = static_cast<unsigned char*>(p);
    return SPH_OK;
}

}  // namespace

extern "C" sph_status sph_sort_keys_static(const uint64_t* keys, int64_t n, uint64_t* sorted_keys,
                                           int32_t* perm, void* stream) {
    if (!keys || !sorted_keys || !perm) return SPH_ERR_INVALID;
    if (n < 1 || n > kMaxKeys) return SPH_ERR_INVALID;
    // An error left pending by earlier, unrelated work on this thread is not
    // this sort's: report it without launching, and without clearing it.
    if (cudaPeekAtLastError() != cudaSuccess) return SPH_ERR_CUDA;
    unsigned char* base = nullptr;
    sph_status st = scratch_for_current_device(&base);
    if (st != SPH_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int nn = (int)n;
    const int nblk = (nn + kTile - 1) / kTile;
    unsigned long long* kb = reinterpret_cast<unsigned long long*>(base + kOffKeys);
    unsigned* vb = reinterpret_cast<unsigned*>(base + kOffVals);
    unsigned* counts = reinterpret_cast<unsigned*>(base + kOffCounts);
    unsigned* cscan = reinterpret_cast<unsigned*>(base + kOffScan);
    unsigned* tmp = reinterpret_cast<unsigned*>(base + kOffTmp);
    // Every scratch word a pass reads is written earlier in the same pass
    // (histograms, their scan, the scattered keys), so nothing left over from
    // an earlier call is read and nothing needs clearing.
    unsigned long long* ka = reinterpret_cast<unsigned long long*>(sorted_keys);
    unsigned* va = reinterpret_cast<unsigned*>(perm);
    if (cudaMemcpyAsync(ka, keys, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return SPH_ERR_CUDA;
    sph::k_iota<<<(nn + 255) / 256, 256, 0, s>>>(perm, nn);
    if (cudaGetLastError() != cudaSuccess) return SPH_ERR_CUDA;
    unsigned launches = 0;
    // 8 passes of 8 bits over all 64 key bits: an even count, so the result
    // ends in the caller's buffers. Each launch is checked as it is queued, and
    // the first failure stops the sort.
    for (int shift = 0; shift < 64; shift += 8) {
        sph::k_rs_hist<<<nblk, 256, 0, s>>>(ka, nn, shift, counts, nblk);
        if (cudaGetLastError() != cudaSuccess) return SPH_ERR_CUDA;
        sph::scan_exclusive<uint32_t>(counts, 256 * nblk, cscan, tmp, s, &launches);
        if (cudaGetLastError() != cudaSuccess) return SPH_ERR_CUDA;
        sph::k_rs_scatter<<<nblk, 256, 0, s>>>(ka, va, kb, vb, nn, shift, cscan, counts, nblk);
        if (cudaGetLastError() != cudaSuccess) return SPH_ERR_CUDA;
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    return SPH_OK;
}
