// common.cuh -- shared device/host helpers of libgi (sm_103a).
//
// Data layout (all device memory, caller-owned unless noted):
//   rec[g]        8 x f32 = (mx, my, m11, m21, m22, c'r, c'g, c'b) with
//                 [[m11, 0], [m21, m22]] = sqrt(log2(e)/2) L^-1, i.e.
//                 m11 = k/l1, m21 = -k l2/(l1 l3), m22 = k/l3, k = sqrt(log2(e)/2):
//                 z1 = m11 dx, z2 = m21 dx + m22 dy and
//                 exp(-sigma) = exp2(-(z1^2 + z2^2)) (sigma = 1/2 d^T Sigma^-1 d).
//   rect[g]       int4 (tx0, ty0, tx1, ty1), image-local tile coordinates.
//   cnt[g]        int32 number of tiles in rect (0 = culled).
//   pair_off[g]   int64 exclusive prefix of cnt: index of g's first pair in
//                 emission order (row-major tiles of the rect).
//   keys / ids    u32 global tile id / Gaussian id of each pair, sorted by
//                 tile, ascending Gaussian id inside a tile.
//   rec_binned[k] the record of ids[k] (tile lists contiguous in memory).
//   ranges[t]     int2 [begin, end) of global tile t in the sorted pairs.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "../../include/gi.h"

namespace gi {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kSqrtHalfLog2e = 0.84932180028801904272f;  // sqrt(log2(e) / 2)
constexpr int kMaxCapacityLog2 = 30;  // pair indices fit the 30-bit look-back field
constexpr int64_t kMaxCapacity = (int64_t(1) << kMaxCapacityLog2) - 1;

// Device-side error bits, OR-ed into a status word by kernels.
enum : uint32_t {
    kErrCapacity = 1u << 0,  // more pairs than capacity
    kErrTimeout = 1u << 1,   // a bounded wait gave up
    kErrBounds = 1u << 2,    // an index check failed
};

// Look-back words: 2 flag bits (aggregate / inclusive prefix) over a 30-bit
// value; spins on an unpublished word are bounded by kSpinLimit.
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagPre = 2u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1;
constexpr uint32_t kSpinLimit = 1u << 20;      // look-back spins (>= 64 ns each after the first 16)
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // bounded mbarrier waits: 1 s

// Per-image descriptor. Pixels of image b live at pix_base + y*W + x.
struct ImgDesc {
    int32_t W, H, tw, th;
    int32_t tile_base;   // first global tile id
    int32_t gauss_base;  // first Gaussian index
    int64_t pix_base;    // first pixel index
};

// Codec fine-tuning state (Sec. 3.3): the render sees FP16 positions, the
// b-bit quantised Cholesky vector and the RVQ colour; bits == 0 is off.
constexpr int kCodecMaxStages = 4;
constexpr int kCodecMaxSize = 256;     // entries per codebook
constexpr int kCodecMaxEntries = 512;  // entries over all stages
constexpr int kCodecMaxVals = 6 + kCodecMaxEntries * 4 + 1;
struct CodecCfg {
    int32_t bits;          // b (1..8); 0: no codec
    int32_t stages, size;  // M, B
    float qp;              // 2^b - 1
    float decay, eps;      // EMA decay and Laplace smoothing of the codebook update
    float* gb;             // [6] gamma[3], beta[3]; followed by the optimiser state [4][6]
    float* codebooks;      // [M][B][3]
    double* ema_count;     // [M][B]
    double* ema_total;     // [M][B][3]
    uchar4* codes;         // [N] quantiser codes (x, y, z; w = 0)
    uint16_t* means16;     // [N][2] binary16 bits of the rendered positions (nullable)
    uint8_t* idx;          // [M][N] RVQ indices
    double* part;          // [nvals][blocks of the reduction] per-block partial sums
    double* tot;           // [nvals] their totals
    unsigned* ticket;      // last-block election of the update kernel (0 between launches)
    double* out;           // [7]: commitment loss L_c, dL/dgamma[3], dL/dbeta[3]
};

__device__ __forceinline__ int codec_nvals(const CodecCfg& c) { return 6 + c.stages * c.size * 4 + 1; }

// Separate opacity (the basic 2D Gaussian of Sec. 3.1, Table 3's "w/o M"):
// o = sigmoid(logit) per Gaussian. mode 1: accumulated summation with
// c' = c o (Eq. 5); mode 2: sorted alpha-blending (Eq. 3-4, "w/o AR").
struct OpacCfg {
    int32_t mode;        // 0: merged colour (c' stored directly)
    float* logit;        // [N] parameter
    float* o;            // [N] sigmoid(logit) of the last formation
    float* m;            // [N] optimiser state
    float* v;
    float* n;            // [N] Adan only
    float* gp;           // [N] Adan only
    float* grad;         // [N] dL/dlogit of the last step
    float* partial;      // [capacity] mode 2: per-pair sum of dL/dalpha w
    int32_t* n_last;     // [pixels] mode 2: list entries each pixel walked
};

// 3D GS's alpha-blending thresholds: skip alpha < 1/255, clamp alpha to
// 0.99, stop before the transmittance falls below 1e-4.
constexpr float kBlendAlphaMin = 1.0f / 255.0f;
constexpr float kBlendAlphaMax = 0.99f;
constexpr float kBlendTMin = 1e-4f;

// Either a single image (by value) or nimg > 1 images in device memory.
struct Batch {
    ImgDesc one;
    const ImgDesc* many;
    int32_t nimg;
    int32_t tile;         // tile edge T (8, 16 or 32)
    int32_t total_tiles;  // sum of tw*th
    int32_t total_gauss;  // sum of n
    int32_t split;        // render: warp groups sharing one tile's list (0 = default for the tile edge)
    int32_t param_mode;   // 0: pixel-space parameters; 1: raw parameters of App. C.1 (tanh positions,
                          //    Cholesky diagonal + 0.5), formation maps them to pixel space
    int32_t cov_mode;     // 0: covariance slots hold the Cholesky vector (l1, l2, l3);
                          // 1: rotation-scaling form (theta, s1, s2), Sigma = (R S)(R S)^T
    CodecCfg codec;       // quantisation-aware fine-tuning (fit contexts only)
    OpacCfg opac;         // separate opacity / alpha-blending (fit contexts only)
};

// b-bit asymmetric quantiser of one Cholesky component (Sec. 3.3, LSQ+ form):
// x = (l - beta) / gamma, code = round(clamp(x, 0, qp)) half to even,
// l_bar = code * gamma + beta, every operation rounded once (no contraction).
__device__ __forceinline__ float lsq_quant(float l, float gamma, float beta, float qp, float& x, float& code) {
    x = __fdiv_rn(__fsub_rn(l, beta), gamma);
    const float xc = x < 0.f ? 0.f : (x > qp ? qp : x);
    code = rintf(xc);
    return __fadd_rn(__fmul_rn(code, gamma), beta);
}

// One greedy RVQ stage (Sec. 3.3, Eq. 10): the entry of cb [size][3] nearest to
// r, distances ((e0^2 + e1^2) + e2^2) in FP32 with one rounding per operation,
// scanning upward and moving only on a strictly smaller distance.
__device__ __forceinline__ float rvq_dist(const float* __restrict__ e, float r0, float r1, float r2) {
    const float e0 = __fsub_rn(e[0], r0), e1 = __fsub_rn(e[1], r1), e2 = __fsub_rn(e[2], r2);
    return __fadd_rn(__fadd_rn(__fmul_rn(e0, e0), __fmul_rn(e1, e1)), __fmul_rn(e2, e2));
}

__device__ __forceinline__ int rvq_pick(const float* __restrict__ cb, int size, float r0, float r1, float r2) {
    int best = 0;
    float bd = rvq_dist(cb, r0, r1, r2);
    for (int j = 1; j < size; ++j) {
        const float d = rvq_dist(cb + 3 * j, r0, r1, r2);
        if (d < bd) {
            bd = d;
            best = j;
        }
    }
    return best;
}

__device__ __forceinline__ ImgDesc img_desc(const Batch& b, int i) {
    return b.nimg == 1 ? b.one : b.many[i];
}

// Image owning Gaussian g (binary search over gauss_base).
__device__ __forceinline__ int image_of_gauss(const Batch& b, int g) {
    if (b.nimg == 1) return 0;
    int lo = 0, hi = b.nimg - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (b.many[mid].gauss_base <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Image owning global tile t (binary search over tile_base).
__device__ __forceinline__ int image_of_tile(const Batch& b, int t) {
    if (b.nimg == 1) return 0;
    int lo = 0, hi = b.nimg - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (b.many[mid].tile_base <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------

// 2^x on the SFU (MUFU.EX2), flush-to-zero of denormal results.
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Look-back words carry their flag and value in one 32-bit word and readers
// use nothing else a publisher wrote, so a relaxed (coherent, single-copy
// atomic) store suffices and avoids the fence of a release.
__device__ __forceinline__ void st_relaxed_u32(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Bounded wait on an mbarrier phase; returns false if it gave up.
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for phase `parity` of the mbarrier; gives up (returns false) once
// limit_ns of global time have passed, so a copy that never lands cannot
// hang the kernel.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns = kWaitLimitNs) {
    const uint32_t addr = smem_addr(bar);
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 15u) == 15u && globaltimer_ns() - t0 > limit_ns) return false;
    }
}

// 1-D bulk copy global -> shared (TMA unit), completion counted on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// 16-byte asynchronous global -> shared copy through L2 only (cp.async.cg);
// both addresses 16-byte aligned. cp_async_wait_all() waits for every copy
// the thread issued.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void flag_error(uint32_t* status, uint32_t bits) {
    if (status) atomicOr(status, bits);
}

// Programmatic dependent launch: every kernel of the library starts with this
// wait, so a kernel launched with launch_pdl may be scheduled while its
// predecessor drains, and still sees all of the predecessor's results (and
// no predecessor still reads what it overwrites). A no-op for plain launches.
// Extra index checks of the bounds-checking build (-DGI_CHECK_BOUNDS):
// gi_in_bounds(cond, status) raises kErrBounds and returns false when cond
// fails; in the release build it is constant true and compiles away.
__device__ __forceinline__ bool gi_in_bounds(bool cond, uint32_t* status) {
#ifdef GI_CHECK_BOUNDS
    if (!cond) flag_error(status, kErrBounds);
    return cond;
#else
    (void)status;
    (void)cond;
    return true;
#endif
}

// Host-side NVTX range for the lifetime of the object (shows each call and
// each stage of a fit step on a profiler timeline; free when no tool is
// attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};


template <typename Tv>
__device__ __forceinline__ Tv warp_incl_scan(Tv v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        Tv u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

template <typename Tv>
__device__ __forceinline__ Tv warp_sum(Tv v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Inclusive scan over the block (blockDim.x a multiple of 32, <= 1024).
template <typename Tv>
__device__ Tv block_incl_scan(Tv v, Tv* s_warp /*[32]*/) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_incl_scan(v);
    if (lane == 31) s_warp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        Tv w = lane < nw ? s_warp[lane] : Tv(0);
        w = warp_incl_scan(w);
        if (lane < nw) s_warp[lane] = w;
    }
    __syncthreads();
    if (warp > 0) v += s_warp[warp - 1];
    __syncthreads();
    return v;
}

template <typename Tv>
__device__ Tv block_sum(Tv v, Tv* s_warp /*[32]*/) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    if (lane == 0) s_warp[warp] = v;
    __syncthreads();
    Tv r = Tv(0);
    if (warp == 0) {
        r = lane < nw ? s_warp[lane] : Tv(0);
        r = warp_sum(r);
        if (lane == 0) s_warp[0] = r;
    }
    __syncthreads();
    r = s_warp[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// 32-byte global accesses (one 256-bit instruction); p 32-byte aligned.
__device__ __forceinline__ void st_global_v8(void* p, float4 a, float4 b) {
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(a.x), "f"(a.y), "f"(a.z),
                 "f"(a.w), "f"(b.x), "f"(b.y), "f"(b.z), "f"(b.w)
                 : "memory");
}
__device__ __forceinline__ void ld_global_v8(const void* p, float4& a, float4& b) {
    asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
                 : "l"(p));
}

// Launch with the programmatic-stream-serialisation attribute (the launch
// overlaps the previous kernel's tail; captured into graphs as a
// programmatic dependency edge).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

}  // namespace gi

// Host-side launch check: returns GI_ERR_CUDA from the enclosing function.
#define GI_CUDA_TRY(expr)                                      \
    do {                                                       \
        cudaError_t e_ = (expr);                               \
        if (e_ != cudaSuccess) return gi::set_cuda_error(e_, #expr); \
    } while (0)
