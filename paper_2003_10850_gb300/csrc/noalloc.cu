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
#include <mutex>

#include "internal.cuh"

namespace sph {
// kernels of the grid build (grid.cu), reused unchanged
__global__ void k_rs_hist(const unsigned long long* keys, int n, int shift, unsigned* counts, int nblk);
__global__ void k_rs_scatter(const unsigned long long* kin, const unsigned* vin, unsigned long long* kout,
                             unsigned* vout, int n, int shift, const unsigned* offs, int nblk);
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
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_dev[kMaxDevices] = {};

// Once per device, with that device current: look up the array's device address.
sph_status scratch_for_current_device(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SPH_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) return SPH_ERR_CUDA;
        g_scratch_dev[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_dev[dev];
    return SPH_OK;
}

}  // namespace

extern "C" sph_status sph_sort_keys_static(const uint64_t* keys, int64_t n, uint64_t* sorted_keys,
                                           int32_t* perm, void* stream) {
    if (!keys || !sorted_keys || !perm) return SPH_ERR_INVALID;
    if (n < 1 || n > kMaxKeys) return SPH_ERR_INVALID;
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
    unsigned launches = 0;
    // 8 passes of 8 bits over the 63 key bits: an even count, so the result
    // ends in the caller's buffers
    for (int shift = 0; shift < 63; shift += 8) {
        sph::k_rs_hist<<<nblk, 256, 0, s>>>(ka, nn, shift, counts, nblk);
        sph::scan_exclusive<uint32_t>(counts, 256 * nblk, cscan, tmp, s, &launches);
        sph::k_rs_scatter<<<nblk, 256, 0, s>>>(ka, va, kb, vb, nn, shift, cscan, nblk);
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (cudaGetLastError() != cudaSuccess) return SPH_ERR_CUDA;
    return SPH_OK;
}
