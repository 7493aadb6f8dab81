// selftest.cu -- fic_wait_selftest: the bounded mbarrier wait that every
// tcgen05 kernel of the library uses (tc_common.cuh), run on its own so that
// its expiry path can be checked without a fault.
//
// A one-warp kernel initialises a shared-memory mbarrier that expects one
// arrival.  With `complete` set, one thread arrives and phase 0 completes;
// otherwise nothing ever arrives.  Every lane then waits for phase 0 with the
// kernels' warp-uniform bounded wait.  When the cycle limit passes, the wait
// records a timeout in the error word and returns false, the kernel exits,
// and the host reports FIC_ETIMEOUT, as an encode does; the context stays
// usable.
//
// The error word is a file-scope device variable shared by all calls, so
// calls that overlap on the GPU race; each call clears it first.
#include <cstdint>

#include "common.cuh"
#include "engine.h"
#include "fic.h"
#include "tc_common.cuh"

namespace fic {
namespace {

__device__ int g_wait_err;  // kErrTimeout when the wait gave up
__device__ int g_wait_ok;   // 1 when every lane saw the phase complete

__global__ void __launch_bounds__(32) wait_selftest_kernel(int complete, long long limit)
{
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = tc::smem_u32(&bar);
    if (threadIdx.x == 0) {
        tc::mbar_init(b, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (complete && threadIdx.x == 0) tc::mbar_arrive(b);
    const bool ok = tc::mbar_wait_warp(b, 0, &g_wait_err, limit);
    if (threadIdx.x == 0) g_wait_ok = ok ? 1 : 0;
}

int require_sm103()
{
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FIC_ENODEV;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
        return FIC_ENODEV;
    return (major == 10 && minor == 3) ? FIC_OK : FIC_ENODEV;
}

}  // namespace
}  // namespace fic

extern "C" int fic_wait_selftest(int complete, int64_t limit_cycles, void* stream)
{
    using namespace fic;
    if (limit_cycles < 1 || limit_cycles > FIC_SELFTEST_MAX_CYCLES) return FIC_EINVAL;
    const int dst = require_sm103();
    if (dst) return dst;
    cudaStream_t s = (cudaStream_t)stream;
    const int zero = 0;
    FIC_TRY(cudaMemcpyToSymbolAsync(g_wait_err, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    FIC_TRY(cudaMemcpyToSymbolAsync(g_wait_ok, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    wait_selftest_kernel<<<1, 32, 0, s>>>(complete ? 1 : 0, (long long)limit_cycles);
    FIC_TRY(cudaGetLastError());
    int err = 0, ok = 0;
    FIC_TRY(cudaMemcpyFromSymbolAsync(&err, g_wait_err, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    FIC_TRY(cudaMemcpyFromSymbolAsync(&ok, g_wait_ok, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    FIC_TRY(cudaStreamSynchronize(s));
    if (err == kErrTimeout) return FIC_ETIMEOUT;
    return ok ? FIC_OK : FIC_ECUDA;
}
