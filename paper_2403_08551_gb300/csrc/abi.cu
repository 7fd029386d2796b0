// abi.cu -- extern "C" entry points of libgi for the per-stage operations:
// validation, workspace carve-up and launches. See include/gi.h.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "kernels.cuh"

namespace gi {

namespace {
thread_local char t_err[512] = "";
__device__ uint32_t g_dev_status;

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

bool valid_tile(int t) { return t == 8 || t == 16 || t == 32; }

gi_status check_image(const gi_image& img, const char* fn) {
    if (img.width <= 0 || img.height <= 0 || !valid_tile(img.tile))
        return set_error(GI_ERR_INVALID_ARG, "%s: bad image %dx%d tile %d (tile must be 8, 16 or 32)", fn,
                         img.width, img.height, img.tile);
    const int64_t tw = (img.width + img.tile - 1) / img.tile, th = (img.height + img.tile - 1) / img.tile;
    if (tw * th >= (int64_t(1) << 30))
        return set_error(GI_ERR_INVALID_ARG, "%s: too many tiles (%lld)", fn, (long long)(tw * th));
    return GI_OK;
}

Batch single(const gi_image& img, int32_t n) {
    Batch b{};
    const int tw = (img.width + img.tile - 1) / img.tile, th = (img.height + img.tile - 1) / img.tile;
    b.one = ImgDesc{img.width, img.height, tw, th, 0, 0, 0};
    b.many = nullptr;
    b.nimg = 1;
    b.tile = img.tile;
    b.total_tiles = tw * th;
    b.total_gauss = n;
    return b;
}

#define GI_REQUIRE(cond, ...)                                   \
    do {                                                        \
        if (!(cond)) return set_error(GI_ERR_INVALID_ARG, __VA_ARGS__); \
    } while (0)

}  // namespace

gi_status set_error(gi_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_err, sizeof(t_err), fmt, ap);
    va_end(ap);
    return st;
}

gi_status set_cuda_error(cudaError_t e, const char* what) {
    snprintf(t_err, sizeof(t_err), "%s: CUDA error %d (%s)", what, (int)e, cudaGetErrorString(e));
    return GI_ERR_CUDA;
}

cudaError_t smem_optin(const void* kernel, int bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> done;  // (kernel, device) -> limit set
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    int& have = done[{kernel, dev}];
    if (have >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) have = bytes;
    return e;
}

int sm_count() {
    static std::mutex mu;
    static std::map<int, int> cached;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    std::lock_guard<std::mutex> lk(mu);
    int& v = cached[dev];
    if (v <= 0 && (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)) {
        v = 0;
        return 152;
    }
    return v;
}

uint32_t* device_status() {
    static uint32_t* cache[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!cache[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_dev_status) != cudaSuccess) return nullptr;
        cache[dev] = static_cast<uint32_t*>(p);
    }
    return cache[dev];
}

}  // namespace gi

using namespace gi;

extern "C" {

int32_t gi_abi_version(void) { return 8; }

const char* gi_last_error(void) { return t_err; }

const char* gi_status_string(int32_t st) {
    switch (st) {
        case GI_OK: return "GI_OK";
        case GI_ERR_INVALID_ARG: return "GI_ERR_INVALID_ARG";
        case GI_ERR_CUDA: return "GI_ERR_CUDA";
        case GI_ERR_CAPACITY: return "GI_ERR_CAPACITY";
        case GI_ERR_TIMEOUT: return "GI_ERR_TIMEOUT";
        case GI_ERR_UNSUPPORTED: return "GI_ERR_UNSUPPORTED";
        case GI_ERR_NO_MEMORY: return "GI_ERR_NO_MEMORY";
        default: return "GI_ERR_UNKNOWN";
    }
}

gi_status gi_device_errors(uint32_t* bits, int32_t clear, gi_stream stream) {
    GI_REQUIRE(bits, "gi_device_errors: bits is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint32_t* st = device_status();
    if (!st) return set_error(GI_ERR_CUDA, "gi_device_errors: no device status word");
    uint32_t v = 0;
    GI_CUDA_TRY(cudaStreamSynchronize(s));
    GI_CUDA_TRY(cudaMemcpy(&v, st, sizeof(v), cudaMemcpyDeviceToHost));
    if (clear) GI_CUDA_TRY(cudaMemset(st, 0, sizeof(uint32_t)));
    *bits = v;
    return GI_OK;
}

gi_status gi_project(const float* means, const float* chol, const float* color, int32_t n, gi_image img,
                     float* rec, int32_t* rect, int32_t* cnt, gi_stream stream) {
    NvtxRange nvtx_("gi_project");
    gi_status st = check_image(img, "gi_project");
    if (st != GI_OK) return st;
    GI_REQUIRE(n >= 0, "gi_project: n < 0");
    if (n == 0) return GI_OK;
    GI_REQUIRE(means && chol && color && rec && rect && cnt, "gi_project: NULL pointer");
    GI_REQUIRE(aligned(rec, 16) && aligned(rect, 16) && aligned(means, 4) && aligned(chol, 4) &&
                   aligned(color, 4) && aligned(cnt, 4),
               "gi_project: misaligned pointer");
    const Batch B = single(img, n);
    ZeroJob zj{};
    cudaError_t e = launch_project(params_soa(means, chol, color), B, reinterpret_cast<float4*>(rec),
                                   reinterpret_cast<int4*>(rect), cnt, nullptr, zj,
                                   reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return set_cuda_error(e, "gi_project");
    return GI_OK;
}

gi_status gi_bin_workspace_size(int32_t n, gi_image img, int64_t capacity, size_t* bytes) {
    gi_status st = check_image(img, "gi_bin_workspace_size");
    if (st != GI_OK) return st;
    GI_REQUIRE(bytes, "gi_bin_workspace_size: bytes is NULL");
    GI_REQUIRE(n >= 0 && capacity >= 1 && capacity <= kMaxCapacity,
               "gi_bin_workspace_size: bad n (%d) or capacity (%lld)", n, (long long)capacity);
    const Batch B = single(img, n);
    *bytes = bin_ws_layout(nullptr, n, capacity, B.total_tiles).bytes;
    return GI_OK;
}

gi_status gi_bin_tiles(const int32_t* rect, const int32_t* cnt, const float* rec, int32_t n, gi_image img,
                       int64_t capacity, void* ws, size_t ws_bytes, uint32_t* keys, uint32_t* ids,
                       int32_t* ranges, float* rec_binned, int64_t* pair_off, int64_t* k_dev,
                       gi_stream stream) {
    NvtxRange nvtx_("gi_bin_tiles");
    gi_status st = check_image(img, "gi_bin_tiles");
    if (st != GI_OK) return st;
    GI_REQUIRE(n >= 0, "gi_bin_tiles: n < 0");
    GI_REQUIRE(capacity >= 1 && capacity <= kMaxCapacity, "gi_bin_tiles: capacity %lld outside [1, 2^30)",
               (long long)capacity);
    GI_REQUIRE(ws && keys && ids && ranges && pair_off && k_dev && (n == 0 || (rect && cnt)),
               "gi_bin_tiles: NULL pointer");
    GI_REQUIRE(!rec_binned || rec || n == 0, "gi_bin_tiles: rec_binned needs rec");
    GI_REQUIRE(aligned(ws, 256), "gi_bin_tiles: workspace must be 256-byte aligned");
    GI_REQUIRE(aligned(ranges, 16) && aligned(keys, 4) && aligned(ids, 4) && aligned(pair_off, 8) &&
                   aligned(k_dev, 8) && (!rec || aligned(rec, 16)) && (!rec_binned || aligned(rec_binned, 16)) &&
                   (!rect || aligned(rect, 16)),
               "gi_bin_tiles: misaligned pointer");
    const Batch B = single(img, n);
    const BinWs w = bin_ws_layout(ws, n, capacity, B.total_tiles);
    GI_REQUIRE(ws_bytes >= w.bytes, "gi_bin_tiles: workspace %zu bytes < %zu needed", ws_bytes, w.bytes);
    cudaError_t e = launch_bin(reinterpret_cast<const int4*>(rect), cnt, reinterpret_cast<const float4*>(rec), B,
                               capacity, w, false, keys, ids, reinterpret_cast<int2*>(ranges),
                               reinterpret_cast<float4*>(rec_binned), nullptr, pair_off, k_dev, nullptr, device_status(),
                               reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return set_cuda_error(e, "gi_bin_tiles");
    return GI_OK;
}

gi_status gi_render(const float* rec_binned, const int32_t* ranges, gi_image img, const float* target, float* out,
                    float* dl_dout, double* loss_sum, gi_stream stream) {
    NvtxRange nvtx_("gi_render");
    gi_status st = check_image(img, "gi_render");
    if (st != GI_OK) return st;
    GI_REQUIRE(rec_binned && ranges && out, "gi_render: NULL pointer");
    GI_REQUIRE(!dl_dout || target, "gi_render: dl_dout needs target");
    GI_REQUIRE(!loss_sum || target, "gi_render: loss_sum needs target");
    GI_REQUIRE(aligned(rec_binned, 16) && aligned(ranges, 8) && aligned(out, 4) && (!target || aligned(target, 4)) &&
                   (!dl_dout || aligned(dl_dout, 4)) && (!loss_sum || aligned(loss_sum, 8)),
               "gi_render: misaligned pointer");
    const Batch B = single(img, 0);
    cudaError_t e = launch_render(reinterpret_cast<const float4*>(rec_binned), reinterpret_cast<const int2*>(ranges),
                                  B, target, out, dl_dout, nullptr, loss_sum, nullptr, device_status(),
                                  reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return set_cuda_error(e, "gi_render");
    return GI_OK;
}

gi_status gi_backward_workspace_size(int32_t n, gi_image img, int64_t capacity, size_t* bytes) {
    gi_status st = check_image(img, "gi_backward_workspace_size");
    if (st != GI_OK) return st;
    GI_REQUIRE(bytes, "gi_backward_workspace_size: bytes is NULL");
    GI_REQUIRE(n >= 0 && capacity >= 1 && capacity <= kMaxCapacity, "gi_backward_workspace_size: bad n or capacity");
    const Batch B = single(img, n);
    const size_t part = ((size_t)capacity * 32 + 255) / 256 * 256;
    const size_t dl = ((size_t)B.total_tiles * img.tile * img.tile * 12 + 255) / 256 * 256;
    const size_t emit = ((size_t)capacity * 4 + 255) / 256 * 256;
    *bytes = part + dl + emit;
    return GI_OK;
}

gi_status gi_render_backward(const float* rec_binned, const uint32_t* keys, const uint32_t* ids,
                             const int32_t* ranges, const int32_t* rect, const int32_t* cnt,
                             const int64_t* pair_off, const int64_t* k_dev, const float* chol, int32_t n,
                             gi_image img, int64_t capacity, const float* dl_dout, void* ws, size_t ws_bytes,
                             float* g_means, float* g_chol, float* g_color, float* g_conic, gi_stream stream) {
    NvtxRange nvtx_("gi_render_backward");
    gi_status st = check_image(img, "gi_render_backward");
    if (st != GI_OK) return st;
    GI_REQUIRE(n >= 0, "gi_render_backward: n < 0");
    GI_REQUIRE(capacity >= 1 && capacity <= kMaxCapacity, "gi_render_backward: bad capacity");
    (void)ranges;
    if (n == 0) return GI_OK;
    GI_REQUIRE(rec_binned && keys && ids && rect && cnt && pair_off && k_dev && chol && dl_dout && ws && g_means &&
                   g_chol && g_color,
               "gi_render_backward: NULL pointer");
    GI_REQUIRE(aligned(rec_binned, 16) && aligned(keys, 16) && aligned(rect, 16) && aligned(ws, 256) &&
                   aligned(pair_off, 8) && aligned(k_dev, 8),
               "gi_render_backward: misaligned pointer");
    size_t need = 0;
    gi_backward_workspace_size(n, img, capacity, &need);
    GI_REQUIRE(ws_bytes >= need, "gi_render_backward: workspace %zu bytes < %zu needed", ws_bytes, need);
    const Batch B = single(img, n);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t part_bytes = ((size_t)capacity * 32 + 255) / 256 * 256;
    const size_t dl_bytes = ((size_t)B.total_tiles * img.tile * img.tile * 12 + 255) / 256 * 256;
    float4* partial = static_cast<float4*>(ws);
    float* dl_tiled = reinterpret_cast<float*>(static_cast<char*>(ws) + part_bytes);
    uint32_t* emit = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + part_bytes + dl_bytes);
    cudaError_t e = launch_pack_dl(dl_dout, B, dl_tiled, s);
    if (e == cudaSuccess)
        e = launch_emit_index(keys, ids, reinterpret_cast<const int4*>(rect), pair_off, B, k_dev, capacity, emit,
                              device_status(), s);
    if (e == cudaSuccess)
        e = launch_backward(reinterpret_cast<const float4*>(rec_binned), keys, emit, dl_tiled, B, k_dev, capacity,
                            partial, device_status(), s);
    if (e == cudaSuccess)
        e = launch_reduce(partial, pair_off, cnt, capacity, n, params_soa(nullptr, chol, nullptr), g_means, g_chol,
                          g_color, g_conic, nullptr, nullptr, nullptr, nullptr, nullptr, B, s);
    if (e != cudaSuccess) return set_cuda_error(e, "gi_render_backward");
    return GI_OK;
}

gi_status gi_vq_decode(const uint16_t* means16, const uint8_t* idx, const float* codebooks, int32_t n,
                       int32_t stages, int32_t cb_size, float* means, float* chol, float* color, gi_stream stream) {
    NvtxRange nvtx_("gi_vq_decode");
    GI_REQUIRE(n >= 0, "gi_vq_decode: n < 0");
    GI_REQUIRE(stages >= 1 && stages <= 8 && cb_size >= 1 && cb_size <= 256,
               "gi_vq_decode: stages must be 1..8 and cb_size 1..256");
    if (n == 0) return GI_OK;
    GI_REQUIRE(means16 && idx && codebooks && means && chol && color, "gi_vq_decode: NULL pointer");
    GI_REQUIRE(aligned(means16, 2) && aligned(codebooks, 4) && aligned(means, 4) && aligned(chol, 4) &&
                   aligned(color, 4),
               "gi_vq_decode: misaligned pointer");
    cudaError_t e = launch_vq_decode(means16, idx, codebooks, n, stages, cb_size, means, chol, color, 0,
                                     reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return set_cuda_error(e, "gi_vq_decode");
    return GI_OK;
}

gi_status gi_codec_decode(const uint16_t* means16, const uint8_t* codes, const float* gamma_beta,
                          const uint8_t* idx, const float* codebooks, int32_t n, int32_t stages, int32_t size,
                          float* means, float* chol, float* color, gi_stream stream) {
    NvtxRange nvtx_("gi_codec_decode");
    GI_REQUIRE(n >= 0, "gi_codec_decode: n < 0");
    GI_REQUIRE(stages >= 1 && stages <= 8 && size >= 1 && size <= 256,
               "gi_codec_decode: stages must be 1..8 and size 1..256");
    GI_REQUIRE(gamma_beta, "gi_codec_decode: NULL gamma_beta");
    if (n == 0) return GI_OK;
    GI_REQUIRE(means16 && codes && idx && codebooks && means && chol && color, "gi_codec_decode: NULL pointer");
    GI_REQUIRE(aligned(means16, 2) && aligned(codes, 4) && aligned(codebooks, 4) && aligned(means, 4) &&
                   aligned(chol, 4) && aligned(color, 4),
               "gi_codec_decode: misaligned pointer");
    cudaError_t e = launch_codec_decode(means16, codes, gamma_beta, idx, codebooks, n, stages, size, means, chol,
                                        color, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return set_cuda_error(e, "gi_codec_decode");
    return GI_OK;
}

}  // extern "C"
