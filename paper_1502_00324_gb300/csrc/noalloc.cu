// noalloc.cu -- fic_domain_pool_noalloc: the domain-pool pipeline (entropy,
// scan, compaction) for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is unavailable or not
// allowed -- inside a host callback or a memory-pool-restricted process, a
// plugin that is handed device buffers by its host application, or a
// program that pre-reserves all device memory at start-up.  Such callers
// pass their own device buffers for the image and the outputs; the
// intermediate arrays (per-position flags, scan positions, scan tile sums,
// the fixed-point q log2 q table, two counters) live in one file-scope static device
// array instead of the library's allocating workspace.
//
// Scratch: FIC_NOALLOC_MAX_POSITIONS (2^20) domain positions, 8,398,592
// bytes (8.0 MiB) per GPU that loads the library, held until the process
// exits.  Every call
// shares it and it keeps the last call's contents, so calls that overlap on
// the GPU (different streams or threads without ordering) race; the counter
// that accumulates is cleared at the start of each call, everything else is
// fully overwritten.
//
// Set-up: every call looks up the array's device address on the current
// device with cudaGetSymbolAddress (a lookup, no allocation).  The first call
// on a device, and the first call after the module was loaded again (a new
// context after cudaDeviceReset, where the address can change), fills the
// table with one kernel launch and waits for it: make that call before any
// stream capture.
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "fic.h"
#include "kernels.h"

namespace fic {
namespace {

constexpr int64_t kMaxPos = FIC_NOALLOC_MAX_POSITIONS;
constexpr int kTableCount = kEntTableCount;  // fixed-point q log2 q
constexpr int64_t kScanWords = (kMaxPos + 4095) / 4096 + 1;

constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kOffFlags = 0;
constexpr size_t kOffPos = align256(kOffFlags + sizeof(uint32_t) * kMaxPos);
constexpr size_t kOffScan = align256(kOffPos + sizeof(uint32_t) * kMaxPos);
constexpr size_t kOffTable = align256(kOffScan + sizeof(uint32_t) * kScanWords);
constexpr size_t kOffTotal = align256(kOffTable + sizeof(long long) * kTableCount);
constexpr size_t kOffNear = kOffTotal + 8;
constexpr size_t kScratchBytes = align256(kOffNear + 8);
static_assert(kScratchBytes == 8398592, "scratch size stated in fic.h");

// The scratch.  In host code this name is a host-side stand-in, not a device
// address: host code must use the address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// The address whose table was filled, per device ordinal.
struct DeviceSlot {
    unsigned char* filled = nullptr;
};
std::mutex g_mu;
DeviceSlot g_slot[64];

bool on_device(const void* p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Scratch address on the current device; the entropy table is filled when
// this address has not been filled before (no allocation).
int setup(cudaStream_t s, unsigned char** base)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return FIC_ENODEV;
    int major = 0, minor = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
        return FIC_ENODEV;
    if (major != 10 || minor != 3) return FIC_ENODEV;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return FIC_ECUDA;
    unsigned char* b = static_cast<unsigned char*>(p);
    std::lock_guard<std::mutex> g(g_mu);
    if (g_slot[dev].filled != b) {
        g_slot[dev].filled = nullptr;
        if (launch_entropy_table(reinterpret_cast<long long*>(b + kOffTable), kTableCount, s) !=
            cudaSuccess)
            return FIC_ECUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return FIC_ECUDA;
        g_slot[dev].filled = b;
    }
    *base = b;
    return FIC_OK;
}

}  // namespace
}  // namespace fic

using namespace fic;

extern "C" int fic_domain_pool_noalloc(const uint8_t* d_img, int N, int B, int L,
                                       double entropy_thresh, uint32_t* d_pool_xy, int64_t cap,
                                       int64_t* dn, double* d_entropy, int64_t* near,
                                       void* stream)
{
    if (!d_img || !dn || N <= 0 || N > 65535 || L < 1 || cap < 0) return FIC_EINVAL;
    if (!(B == 2 || B == 4 || B == 8 || B == 16)) return FIC_EINVAL;
    if (cap > 0 && !d_pool_xy) return FIC_EINVAL;
    const int per = (N >= 2 * B) ? (N - 2 * B) / L + 1 : 0;
    const int64_t npos = (int64_t)per * per;
    if (npos > kMaxPos) return FIC_EINVAL;  // larger than the static scratch
    if (!on_device(d_img) || (d_pool_xy && !on_device(d_pool_xy)) ||
        (d_entropy && !on_device(d_entropy)))
        return FIC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* base = nullptr;
    int st = setup(s, &base);
    if (st) return st;
    uint32_t* flags = reinterpret_cast<uint32_t*>(base + kOffFlags);
    uint32_t* pos = reinterpret_cast<uint32_t*>(base + kOffPos);
    uint32_t* scan = reinterpret_cast<uint32_t*>(base + kOffScan);
    const long long* table = reinterpret_cast<const long long*>(base + kOffTable);
    uint32_t* total = reinterpret_cast<uint32_t*>(base + kOffTotal);
    unsigned long long* nr = reinterpret_cast<unsigned long long*>(base + kOffNear);

    // a negative threshold admits every position (entropy still reported)
    const double thr = entropy_thresh < 0.0 ? -1.0e300 : entropy_thresh;
    if (cudaMemsetAsync(nr, 0, sizeof(unsigned long long), s) != cudaSuccess) return FIC_ECUDA;
    if (cudaMemsetAsync(total, 0, sizeof(uint32_t), s) != cudaSuccess) return FIC_ECUDA;
    if (npos > 0) {
        if (launch_entropy(d_img, N, B, L, per, thr, table, flags, d_entropy, nullptr, nr, s) !=
            cudaSuccess)
            return FIC_ECUDA;
        if (launch_scan(flags, pos, npos, scan, total, s, nullptr) != cudaSuccess)
            return FIC_ECUDA;
    }
    uint32_t h_total = 0;
    unsigned long long h_near = 0;
    if (cudaMemcpyAsync(&h_total, total, sizeof(h_total), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(&h_near, nr, sizeof(h_near), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return FIC_ECUDA;
    *dn = h_total;
    if (near) *near = entropy_thresh < 0.0 ? 0 : (int64_t)h_near;
    if ((int64_t)h_total > cap) return FIC_ECAP;
    if (npos > 0 && h_total > 0) {
        if (launch_pool_scatter(flags, pos, npos, per, L, d_pool_xy, s) != cudaSuccess)
            return FIC_ECUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return FIC_ECUDA;
    }
    return FIC_OK;
}
