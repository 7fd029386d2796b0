// kernels.cuh -- internal launchers shared by the C-ABI (abi.cu) and the
// fit context (fit.cu). Not part of the public ABI.
#pragma once
#include "common.cuh"

namespace gi {

// Parameter access: AoS [n][8] (mx,my,l1,l2,l3,cr,cg,cb) or SoA arrays.
struct ParamsIn {
    const float* means;  // stride ms floats per Gaussian
    const float* chol;   // stride ls
    const float* color;  // stride cs
    int32_t ms, ls, cs;
};

inline ParamsIn params_soa(const float* m, const float* l, const float* c) { return {m, l, c, 2, 3, 3}; }
inline ParamsIn params_aos(const float* p) { return {p, p + 2, p + 5, 8, 8, 8}; }

// Regions zeroed by the projection kernel before binning: p[r] (16-byte
// aligned) holds n32[r] 32-bit words.
struct ZeroJob {
    uint32_t* p[6];
    int64_t n32[6];
};

// Radix plan for the tile keys.
struct RadixPlan {
    int bits;    // total key bits
    int passes;  // LSD passes
    int dbits;   // digit bits per pass (<= kMaxDigitBits)
};
RadixPlan radix_plan(int total_tiles);

constexpr int kProjBlock = 256;        // Gaussians per projection / emit block
constexpr int kSortThreads = 256;      // threads per onesweep block
constexpr int kSortItems = 16;         // keys per thread
constexpr int kMaxDigitBits = 9;       // radix digits of at most 9 bits (512 buckets)
constexpr int kMaxRadix = 1 << kMaxDigitBits;
constexpr int kMaxPasses = 4;          // 31-bit keys at most
constexpr int kHistReplicas = 8;       // copies of each pass's digit histogram (spread the emit's atomics)
constexpr int kSortTile = kSortThreads * kSortItems;  // keys per onesweep block
constexpr int kSortStageBytes = kSortTile * 8;          // keys + values staged in digit order

// Count-matrix binning (bin_cm.cu): chunks of kCmChunk Gaussians; used when
// the batch has at most kCmMaxTiles tiles and chunks x tiles <= kCmMaxCells.
constexpr int kCmChunk = 128;
constexpr int kCmGroupTiles = 16;  // count-matrix column scan: tiles per block
constexpr int kCmMaxTiles = 2048;
constexpr int64_t kCmMaxCells = int64_t(1) << 20;
bool cm_applies(int64_t n, int total_tiles);

// Binning workspace carve-up. [zero, zero + zero_words) holds every buffer
// that must be zero before a binning pass. Radix path: keys_tmp, vals_tmp,
// hist [passes][kHistReplicas][kMaxRadix], lookback [passes][sort_blocks][kMaxRadix]. Count-matrix path: cm
// [chunks][tiles], chunk_sum [chunks], tile_tot [tiles] (column totals).
struct BinWs {
    bool cm_path;
    int64_t* blk_sum;     // [ceil(n / kProjBlock)]
    uint32_t* keys_tmp;   // [capacity]          (radix)
    uint32_t* vals_tmp;   // [capacity]          (radix)
    uint32_t* owner;      // [capacity] Gaussian of each emission index (radix, optional: then the
                          //            sort carries the emission index instead of the Gaussian)
    uint32_t* cm;         // [chunks][tiles]     (count matrix)
    uint32_t* chunk_sum;  // [chunks]            (count matrix)
    uint32_t* tile_tot;   // [tiles]             (count matrix: column totals, 16-byte aligned)
    uint32_t* zero;
    int64_t zero_words;
    uint32_t* hist;       // [passes][kHistReplicas][kMaxRadix] (radix)
    uint64_t* blk_lb;     // [ceil(n / kProjBlock)] published block prefixes of the key emission (radix)
    uint32_t* lookback;
    uint32_t* tickets;    // [4]
    size_t bytes;
};
BinWs bin_ws_layout(void* base, int64_t n, int64_t capacity, int total_tiles, bool with_owner = true);

// Launchers (stream-ordered, no host synchronisation).
// With cm != null (count-matrix binning to follow) the projection also
// writes the count-matrix rows and chunk totals of its Gaussians.
cudaError_t launch_project(const ParamsIn& P, const Batch& B, float4* rec, int4* rect, int32_t* cnt,
                           int64_t* blk_sum, const ZeroJob& zj, cudaStream_t s, uint32_t* cm = nullptr,
                           uint32_t* chunk_sum = nullptr);
// emit (nullable): [capacity] emission index of each sorted pair.
cudaError_t launch_bin(const int4* rect, const int32_t* cnt, const float4* rec, const Batch& B,
                       int64_t capacity, const BinWs& ws, bool blk_sum_ready, uint32_t* keys,
                       uint32_t* ids, int2* ranges, float4* rec_binned, uint32_t* emit, int64_t* pair_off,
                       int64_t* k_dev, int64_t* k_max, uint32_t* status, cudaStream_t s);

// prepared: the projection already wrote the count-matrix rows and cleared
// the scratch (fit path); otherwise k_count does both.
cudaError_t launch_bin_cm(const int4* rect, const int32_t* cnt, const float4* rec, const Batch& B,
                          int64_t capacity, const BinWs& ws, bool prepared, uint32_t* keys, uint32_t* ids,
                          int2* ranges, float4* rec_binned, uint32_t* emit, int64_t* pair_off, int64_t* k_dev,
                          int64_t* k_max, uint32_t* status, cudaStream_t s);

// Forward render: out (HWC), dL/dC in HWC (dl_hwc) and/or planar per tile
// (dl_tiled: [tile][R,G,B][T*T] f32) and the squared error: with loss_tile
// each tile's sum (a fixed order inside the tile) at loss_tile[t], else
// added to loss_sum (double per image).
// queue (nullable): render with persistent blocks that take tiles from a
// queue ordered by descending list length (built by a one-block kernel
// first); otherwise one block per tile in index order.
struct TileQueue {
    uint32_t* order;  // [tiles]
    uint32_t* head;   // [1]
};
cudaError_t launch_render(const float4* rec_binned, const int2* ranges, const Batch& B,
                          const float* target, float* out, float* dl_hwc, float* dl_tiled,
                          double* loss_sum, double* loss_tile, uint32_t* status, cudaStream_t s,
                          const TileQueue* queue = nullptr);

// Sorted alpha-blending render (Eq. 3-4) and its backward (blend.cu), tile 16
// only; opacity, per-pixel walk lengths and the ninth per-pair sum live in
// B.opac.
cudaError_t launch_render_blend(const float4* rec_binned, const uint32_t* ids, const int2* ranges, const Batch& B,
                                const float* target, float* out, float* dl_tiled, double* loss_sum, uint32_t* status,
                                cudaStream_t s);
cudaError_t launch_backward_blend(const float4* rec_binned, const uint32_t* ids, const int2* ranges, const int4* rect,
                                  const int64_t* pair_off, const Batch& B, const float* out, const float* dl_tiled,
                                  int64_t capacity, float4* partial, uint32_t* status, cudaStream_t s);

// Backward: per-pair partial sums (8 floats per pair at its emission index
// emit[k], written by the binning or by launch_emit_index).
cudaError_t launch_backward(const float4* rec_binned, const uint32_t* keys, const uint32_t* emit,
                            const float* dl_tiled, const Batch& B, const int64_t* k_dev, int64_t capacity,
                            float4* partial, uint32_t* status, cudaStream_t s);
cudaError_t launch_emit_index(const uint32_t* keys, const uint32_t* ids, const int4* rect, const int64_t* pair_off,
                              const Batch& B, const int64_t* k_dev, int64_t capacity, uint32_t* emit,
                              uint32_t* status, cudaStream_t s);
cudaError_t launch_pack_dl(const float* dl_hwc, const Batch& B, float* dl_tiled, cudaStream_t s);

struct AdamCfg {
    float lr[3];  // means, chol, color
    float beta1, beta2, eps;
    int32_t* step;  // device counter (1-based step of the update being made = *step + 1)
    uint32_t* done; // device counter for the last-block step increment
    int32_t optimizer;       // 0: Adam; 1: Adan (beta1, beta2, beta3 decay m, v, n)
    float beta3;             // Adan
    int32_t lr_halve_every;  // every learning rate halves every this many steps; 0 = never
    float* n;                // Adan: second moment of the extrapolated gradient [N][8]
    float* g_prev;           // Adan: previous gradient [N][8]
    int32_t param_mode;      // 1: params are the raw App. C.1 parameters (chain through the formation)
    int32_t cov_mode;        // 1: covariance parameters are (theta, s1, s2) (chain dSigma -> theta, s1, s2)
};

// Reduce partials per Gaussian, chain conic -> Cholesky; then either write
// gradients (g_means/g_chol/g_color/g_conic, SoA, any may be null) or, when
// adam != null, update AoS params/m/v in place (grads_aos optional).
// Blocks of the per-Gaussian reduction for n Gaussians.
int64_t reduce_blocks(int64_t n);
// With loss_tile (fitting), the reduction also writes each image's squared
// error loss[b] as the sum of its tiles' partials in tile order.
cudaError_t launch_reduce(const float4* partial, const int64_t* pair_off, const int32_t* cnt,
                          int64_t capacity, int32_t n, const ParamsIn& P, float* g_means,
                          float* g_chol, float* g_color, float* g_conic, const AdamCfg* adam,
                          float* params, float* m, float* v, float* grads_aos, const Batch& B,
                          cudaStream_t s, const double* loss_tile = nullptr, double* loss = nullptr);

struct GammaBeta {
    float v[6];  // gamma[3], beta[3]
};
cudaError_t launch_codec_decode(const uint16_t* means16, const uint8_t* codes, const float* gamma_beta,
                                const uint8_t* idx, const float* cb, int32_t n, int32_t stages, int32_t size,
                                float* means, float* chol, float* color, cudaStream_t s);

cudaError_t launch_vq_decode(const uint16_t* means16, const uint8_t* idx, const float* cb, int32_t n,
                             int32_t stages, int32_t cb_size, float* means, float* chol, float* color,
                             int32_t out_stride_aos, cudaStream_t s);

// Per-device error word that kernels OR error bits into.
uint32_t* device_status();
// Raises `kernel`'s dynamic shared-memory limit to at least `bytes` on the
// current device, once per (kernel, device); safe to call from several host
// threads and for several devices in one process.
cudaError_t smem_optin(const void* kernel, int bytes);
// Number of SMs of the current device (cached per device).
int sm_count();
gi_status set_cuda_error(cudaError_t e, const char* what);
gi_status set_error(gi_status st, const char* fmt, ...);

}  // namespace gi
