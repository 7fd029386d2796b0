// noalloc.cu -- tile binning for callers that cannot allocate device memory.
//
// gi_bin_tiles needs a scratch workspace that the caller allocates. Some
// callers have no way to do that: code that runs inside another framework's
// memory pool and is not allowed to call cudaMalloc behind its back, code
// that must not trigger the implicit device synchronisation an allocation can
// cause (a latency-critical loop), or a fixed-budget deployment that reserves
// all memory up front. gi_bin_tiles_noalloc serves them: its scratch lives in
// a fixed-size array in this library's device memory, which every GPU that
// loads the library holds until the process exits.
//
// Properties (also stated in include/gi.h):
//  - No allocation: no cudaMalloc, cudaFree or allocating library routine.
//  - Limits: n <= GI_NOALLOC_MAX_GAUSSIANS and capacity <= GI_NOALLOC_MAX_PAIRS
//    (and the image's tile grid); larger sizes are rejected with
//    GI_ERR_INVALID_ARG before anything is launched.
//  - Shared state: every call on a device uses the same array and the array
//    keeps the previous call's contents; the parts that must start at zero
//    (digit histograms, look-back words, tickets, tile ranges) are cleared by
//    the call itself. Calls whose kernels overlap on the GPU (different
//    streams without ordering between them) race on the array.
//  - Set-up: the first call on each device looks up the array's device
//    address with cudaGetSymbolAddress while that device is current. Make
//    that first call before any stream capture.
#include <mutex>

#include "kernels.cuh"

namespace gi {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(6) << 20;  // 6 MiB per device

// The scratch. In host code this name is only a host-side stand-in for the
// symbol; kernels receive the device address looked up below.
static __device__ __align__(256) unsigned char g_bin_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_addr[64] = {nullptr};

// Device address of g_bin_scratch for the current device (looked up once).
gi_status scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_cuda_error(e, "gi_bin_tiles_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= 64) return set_error(GI_ERR_UNSUPPORTED, "gi_bin_tiles_noalloc: device index %d", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_bin_scratch);
        if (e != cudaSuccess) return set_cuda_error(e, "gi_bin_tiles_noalloc: cudaGetSymbolAddress");
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return GI_OK;
}

bool aligned_to(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace
}  // namespace gi

using namespace gi;

extern "C" gi_status gi_bin_tiles_noalloc(const int32_t* rect, const int32_t* cnt, const float* rec, int32_t n,
                                          gi_image img, int64_t capacity, uint32_t* keys, uint32_t* ids,
                                          int32_t* ranges, float* rec_binned, int64_t* pair_off, int64_t* k_dev,
                                          gi_stream stream) {
    NvtxRange nvtx_("gi_bin_tiles_noalloc");
    if (img.width <= 0 || img.height <= 0 || (img.tile != 8 && img.tile != 16 && img.tile != 32))
        return set_error(GI_ERR_INVALID_ARG, "gi_bin_tiles_noalloc: bad image %dx%d tile %d", img.width,
                         img.height, img.tile);
    if (n < 0 || n > GI_NOALLOC_MAX_GAUSSIANS)
        return set_error(GI_ERR_INVALID_ARG, "gi_bin_tiles_noalloc: n = %d outside [0, %d]", n,
                         GI_NOALLOC_MAX_GAUSSIANS);
    if (capacity < 1 || capacity > GI_NOALLOC_MAX_PAIRS)
        return set_error(GI_ERR_INVALID_ARG, "gi_bin_tiles_noalloc: capacity %lld outside [1, %d]",
                         (long long)capacity, GI_NOALLOC_MAX_PAIRS);
    const int64_t tw = (img.width + img.tile - 1) / img.tile, th = (img.height + img.tile - 1) / img.tile;
    if (tw * th >= (int64_t(1) << 30))
        return set_error(GI_ERR_INVALID_ARG, "gi_bin_tiles_noalloc: too many tiles");
    if (!keys || !ids || !ranges || !pair_off || !k_dev || (n > 0 && (!rect || !cnt)))
        return set_error(GI_ERR_INVALID_ARG, "gi_bin_tiles_noalloc: NULL pointer");
    if (rec_binned && !rec && n > 0) return set_error(GI_ERR_INVALID_ARG, "gi_bin_tiles_noalloc: rec_binned needs rec");
    if (!aligned_to(ranges, 16) || !aligned_to(keys, 4) || !aligned_to(ids, 4) || !aligned_to(pair_off, 8) ||
        !aligned_to(k_dev, 8) || (rec && !aligned_to(rec, 16)) || (rec_binned && !aligned_to(rec_binned, 16)) ||
        (rect && !aligned_to(rect, 16)))
        return set_error(GI_ERR_INVALID_ARG, "gi_bin_tiles_noalloc: misaligned pointer");

    Batch B{};
    B.one = ImgDesc{img.width, img.height, (int32_t)tw, (int32_t)th, 0, 0, 0};
    B.nimg = 1;
    B.tile = img.tile;
    B.total_tiles = (int32_t)(tw * th);
    B.total_gauss = n;
    const size_t need = bin_ws_layout(nullptr, n, capacity, B.total_tiles, false).bytes;
    if (need > kNoAllocScratchBytes)
        return set_error(GI_ERR_INVALID_ARG, "gi_bin_tiles_noalloc: needs %zu scratch bytes, the fixed array has %zu",
                         need, kNoAllocScratchBytes);
    void* base = nullptr;
    gi_status st = scratch_address(&base);
    if (st != GI_OK) return st;
    const BinWs w = bin_ws_layout(base, n, capacity, B.total_tiles, false);
    cudaError_t e = launch_bin(reinterpret_cast<const int4*>(rect), cnt, reinterpret_cast<const float4*>(rec), B,
                               capacity, w, false, keys, ids, reinterpret_cast<int2*>(ranges),
                               reinterpret_cast<float4*>(rec_binned), nullptr, pair_off, k_dev, nullptr, device_status(),
                               reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return set_cuda_error(e, "gi_bin_tiles_noalloc");
    return GI_OK;
}
