// selftest.cu -- exercises the bounded waits of the library on the GPU
// without a fault: one kernel waits on an mbarrier that nothing arrives at
// (the wait of the render's TMA staging), one spins on a flag that nothing
// sets (the pattern of the look-back scans); both must give up after their
// limit and report it, leaving the context usable.
#include "kernels.cuh"

namespace gi {
namespace {

__device__ uint32_t g_selftest_bits;  // private status word of the self-test
__device__ uint32_t g_selftest_flag;  // the flag the spin test waits on; only zeroed, never set

__global__ void k_selftest_mbar(uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const bool arrived = mbar_wait(&bar, 0, limit_ns);  // nothing arrives
    if (!arrived && threadIdx.x == 0) atomicOr(&g_selftest_bits, 1u);
    if (arrived && threadIdx.x == 0) atomicOr(&g_selftest_bits, 4u);  // cannot happen: reported as an error
}

__global__ void k_selftest_spin(const uint32_t* flag, uint64_t limit_ns) {
    const uint64_t t0 = globaltimer_ns();
    uint32_t spins = 0;
    while (ld_relaxed_u32(flag) == 0u) {  // nothing sets the flag
        if (++spins > 16) __nanosleep(64);
        if (globaltimer_ns() - t0 > limit_ns) {
            if (threadIdx.x == 0) atomicOr(&g_selftest_bits, 2u);
            return;
        }
    }
    if (threadIdx.x == 0) atomicOr(&g_selftest_bits, 8u);
}

}  // namespace
}  // namespace gi

using namespace gi;

extern "C" {

gi_status gi_selftest_bounded_waits(uint32_t* observed, int64_t limit_ns, gi_stream stream) {
    NvtxRange nvtx_("gi_selftest_bounded_waits");
    if (!observed || limit_ns <= 0 || limit_ns > 2000000000ll)
        return set_error(GI_ERR_INVALID_ARG, "gi_selftest_bounded_waits: bad argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const uint32_t zero = 0;
    uint32_t* bits = nullptr;
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&bits), g_selftest_bits);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bits, &zero, 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) k_selftest_mbar<<<1, 32, 0, s>>>((uint64_t)limit_ns);
    if (e == cudaSuccess) e = cudaGetLastError();
    uint32_t* flag = nullptr;
    if (e == cudaSuccess) e = cudaGetSymbolAddress(reinterpret_cast<void**>(&flag), g_selftest_flag);
    if (e == cudaSuccess) e = cudaMemcpyAsync(flag, &zero, 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) k_selftest_spin<<<1, 32, 0, s>>>(flag, (uint64_t)limit_ns);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(observed, bits, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_cuda_error(e, "gi_selftest_bounded_waits");
    return GI_OK;
}

}  // extern "C"
