// fit.cu -- image fitting contexts (Sec. 3.4): one step = formation,
// binning, render + L2 loss, backward and an Adam update, for one image or a
// batch of images of different sizes whose tiles share every launch. The
// step is five stream-ordered stages with no host round trip (pair counts
// stay on the device), captured once into a CUDA graph and replayed.
#include <cstring>
#include <new>
#include <vector>

#include "kernels.cuh"

using namespace gi;

struct gi_fit {
    int dev = 0;
    int nimg = 0;
    int64_t N = 0;
    int64_t npix = 0;
    int64_t capacity = 0;
    Batch B{};
    AdamCfg adam{};
    bool use_graph = false;
    bool stage_events = false;
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t render_graph = nullptr;  // forward only (no loss), for gi_fit_render
    cudaGraphExec_t render_exec = nullptr;
    void* arena = nullptr;
    // carved from arena
    ImgDesc* d_desc = nullptr;
    float *params = nullptr, *m = nullptr, *v = nullptr, *grads = nullptr;
    float *targets = nullptr, *out = nullptr;
    const float* target_src = nullptr;  // where the render reads the target (default: targets)
    float4 *rec = nullptr, *rec_binned = nullptr, *partial = nullptr;
    float* dl_tiled = nullptr;
    int4* rect = nullptr;
    int32_t* cnt = nullptr;
    int64_t *pair_off = nullptr, *k_dev = nullptr, *k_max = nullptr;
    uint32_t *keys = nullptr, *ids = nullptr, *emit = nullptr, *done = nullptr;
    int2* ranges = nullptr;
    double* loss = nullptr;
    double* loss_tile = nullptr;  // [tiles] squared error per tile of the last step
    bool use_queue = false;
    TileQueue queue{};
    int32_t* step = nullptr;
    BinWs bws{};
};

namespace {

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

cudaError_t mark(gi_fit* f, int i, cudaStream_t s) {
    if (!f->stage_events) return cudaSuccess;
    // Inside a stream capture an external record becomes an event-record node
    // of the graph, so every replay re-records the event.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(f->ev[i], s, cudaEventRecordExternal)
                                               : cudaEventRecord(f->ev[i], s);
}

// Formation, binning and render. train: also the loss and the planar dL/dC
// for the backward, with stage events; otherwise the image only.
cudaError_t enqueue_forward(gi_fit* f, cudaStream_t s, bool train) {
    ZeroJob zj{};
    zj.p[0] = f->bws.zero;
    zj.n32[0] = f->bws.zero_words;
    zj.p[1] = reinterpret_cast<uint32_t*>(f->ranges);
    zj.n32[1] = (int64_t)f->B.total_tiles * 2;
    if (train) {  // the render-only pass leaves the last step's loss in place
        zj.p[2] = reinterpret_cast<uint32_t*>(f->loss);
        zj.n32[2] = (int64_t)f->nimg * 2;
    }
    cudaError_t e = train ? mark(f, 0, s) : cudaSuccess;
    if (e == cudaSuccess) {
        NvtxRange r("gi:formation");
        e = launch_project(params_aos(f->params), f->B, f->rec, f->rect, f->cnt, f->bws.blk_sum, zj, s, f->bws.cm,
                           f->bws.chunk_sum);
    }
    if (e == cudaSuccess && train) e = mark(f, 1, s);
    if (e == cudaSuccess) {
        NvtxRange r("gi:binning");
        e = launch_bin(f->rect, f->cnt, f->rec, f->B, f->capacity, f->bws, true, f->keys, f->ids, f->ranges,
                       f->rec_binned, f->emit, f->pair_off, f->k_dev, f->k_max, device_status(), s);
    }
    if (e == cudaSuccess && train) e = mark(f, 2, s);
    if (e == cudaSuccess) {
        NvtxRange r("gi:render");
        e = f->B.opac.mode == 2
                ? launch_render_blend(f->rec_binned, f->ids, f->ranges, f->B, train ? f->target_src : nullptr, f->out,
                                      train ? f->dl_tiled : nullptr, train ? f->loss : nullptr, device_status(), s)
                : launch_render(f->rec_binned, f->ranges, f->B, train ? f->target_src : nullptr, f->out, nullptr,
                                train ? f->dl_tiled : nullptr, nullptr, train ? f->loss_tile : nullptr,
                                device_status(), s, f->use_queue ? &f->queue : nullptr);
    }
    if (e == cudaSuccess && train) e = mark(f, 3, s);
    return e;
}

cudaError_t enqueue_step(gi_fit* f, cudaStream_t s) {
    cudaError_t e = enqueue_forward(f, s, true);
    if (e != cudaSuccess) return e;
    {
        NvtxRange r("gi:backward");
        e = f->B.opac.mode == 2
                ? launch_backward_blend(f->rec_binned, f->ids, f->ranges, f->rect, f->pair_off, f->B, f->out,
                                        f->dl_tiled, f->capacity, f->partial, device_status(), s)
                : launch_backward(f->rec_binned, f->keys, f->emit, f->dl_tiled, f->B, f->k_dev, f->capacity,
                                  f->partial, device_status(), s);
    }
    if (e == cudaSuccess) e = mark(f, 4, s);
    if (e == cudaSuccess) {
        NvtxRange r("gi:update");
        e = launch_reduce(f->partial, f->pair_off, f->cnt, f->capacity, (int32_t)f->N, params_aos(f->params),
                          nullptr, nullptr, nullptr, nullptr, &f->adam, f->params, f->m, f->v, f->grads, f->B, s,
                          f->B.opac.mode == 2 ? nullptr : f->loss_tile, f->loss);
    }
    if (e == cudaSuccess) e = mark(f, 5, s);
    return e;
}

void destroy_graphs(gi_fit* f) {
    if (f->exec) cudaGraphExecDestroy(f->exec);
    if (f->graph) cudaGraphDestroy(f->graph);
    if (f->render_exec) cudaGraphExecDestroy(f->render_exec);
    if (f->render_graph) cudaGraphDestroy(f->render_graph);
    f->exec = f->render_exec = nullptr;
    f->graph = f->render_graph = nullptr;
}

// Captures the training step and the forward-only pass into graphs.
cudaError_t capture_graphs(gi_fit* f) {
    cudaError_t e = cudaStreamBeginCapture(f->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t ce = enqueue_step(f, f->cap_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(f->cap_stream, &g);
    f->graph = g;
    if (ce != cudaSuccess) return ce;
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(&f->exec, f->graph, 0);
    if (e != cudaSuccess) return e;
    e = cudaStreamBeginCapture(f->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    ce = enqueue_forward(f, f->cap_stream, false);
    cudaGraph_t rg = nullptr;
    e = cudaStreamEndCapture(f->cap_stream, &rg);
    f->render_graph = rg;
    if (ce != cudaSuccess) return ce;
    if (e != cudaSuccess) return e;
    return cudaGraphInstantiate(&f->render_exec, f->render_graph, 0);
}

void release(gi_fit* f) {
    if (!f) return;
    destroy_graphs(f);
    if (f->cap_stream) cudaStreamDestroy(f->cap_stream);
    for (cudaEvent_t e : f->ev)
        if (e) cudaEventDestroy(e);
    if (f->arena) cudaFree(f->arena);
    delete f;
}

// Checks a fitting descriptor (everything but the capacity).
gi_status check_desc(const gi_fit_desc* d, const char* fn) {
    if (d->n_images < 1 || !d->widths || !d->heights || !d->counts || !d->targets || !d->params)
        return set_error(GI_ERR_INVALID_ARG, "%s: bad image list or NULL buffer", fn);
    if (d->tile != 8 && d->tile != 16 && d->tile != 32)
        return set_error(GI_ERR_INVALID_ARG, "%s: tile must be 8, 16 or 32", fn);
    {
        const int sp = d->render_split;
        const bool ok = sp == 0 || (d->tile == 8 && (sp == 2 || sp == 4)) || (d->tile == 16 && (sp == 4 || sp == 8)) ||
                        (d->tile == 32 && (sp == 1 || sp == 2));
        if (!ok)
            return set_error(GI_ERR_INVALID_ARG, "%s: render_split %d not available for tile %d", fn, sp, d->tile);
    }
    if ((d->param_mode != 0 && d->param_mode != 1) || (d->optimizer != 0 && d->optimizer != 1) ||
        (d->cov_mode != 0 && d->cov_mode != 1) || d->lr_halve_every < 0 ||
        (d->optimizer == 1 && !(d->beta3 >= 0.f && d->beta3 < 1.f)))
        return set_error(GI_ERR_INVALID_ARG, "%s: bad param_mode, cov_mode, optimizer, beta3 or lr_halve_every", fn);
    if ((reinterpret_cast<uintptr_t>(d->params) & 15) != 0)
        return set_error(GI_ERR_INVALID_ARG, "%s: params must be 16-byte aligned", fn);
    if (d->tile_queue != 0 && d->tile_queue != 1) return set_error(GI_ERR_INVALID_ARG, "%s: tile_queue must be 0 or 1", fn);
    const bool codec = d->codec_bits != 0;
    if (d->opacity_mode < 0 || d->opacity_mode > 2 || (d->opacity_mode == 2 && d->tile != 16) ||
        (d->opacity_mode != 0 && (codec || d->cov_mode != 0)))
        return set_error(GI_ERR_INVALID_ARG, "%s: opacity_mode must be 0, 1 or 2 (2 needs tile 16; neither 1 nor 2 "
                                             "combines with the codec or the rotation-scaling form)", fn);
    if (codec) {
        if (d->codec_bits < 1 || d->codec_bits > 8 || d->codec_stages < 1 || d->codec_stages > kCodecMaxStages ||
            d->codec_size < 1 || d->codec_size > kCodecMaxSize || d->codec_stages * d->codec_size > kCodecMaxEntries ||
            !d->codebooks)
            return set_error(GI_ERR_INVALID_ARG, "%s: codec needs bits in [1, 8], stages in [1, %d], size in [1, %d], "
                                                 "stages x size <= %d and codebooks", fn, kCodecMaxStages,
                             kCodecMaxSize, kCodecMaxEntries);
        if (d->n_images != 1 || d->cov_mode != 0)
            return set_error(GI_ERR_INVALID_ARG, "%s: codec fine-tuning takes one image in Cholesky form", fn);
        if (!(d->ema_decay >= 0.f && d->ema_decay < 1.f) || !(d->ema_eps >= 0.f) ||
            !(d->lsq_gamma[0] > 0.f && d->lsq_gamma[1] > 0.f && d->lsq_gamma[2] > 0.f))
            return set_error(GI_ERR_INVALID_ARG, "%s: codec needs ema_decay in [0, 1), ema_eps >= 0 and gamma > 0", fn);
    }
    return GI_OK;
}

// Per-image descriptors of the batch (first tile, Gaussian and pixel of
// each image) and the totals.
gi_status image_table(const gi_fit_desc* d, const char* fn, std::vector<ImgDesc>& desc, int64_t& tiles,
                      int64_t& gauss, int64_t& pix) {
    desc.assign(d->n_images, ImgDesc{});
    tiles = gauss = pix = 0;
    for (int i = 0; i < d->n_images; ++i) {
        const int W = d->widths[i], H = d->heights[i], n = d->counts[i];
        if (W <= 0 || H <= 0 || n < 0) return set_error(GI_ERR_INVALID_ARG, "%s: bad image %d", fn, i);
        const int tw = (W + d->tile - 1) / d->tile, th = (H + d->tile - 1) / d->tile;
        desc[i] = ImgDesc{W, H, tw, th, (int32_t)tiles, (int32_t)gauss, pix};
        tiles += (int64_t)tw * th;
        gauss += n;
        pix += (int64_t)W * H;
    }
    if (tiles >= (int64_t(1) << 30) || gauss >= (int64_t(1) << 31) - 1)
        return set_error(GI_ERR_INVALID_ARG, "%s: batch too large", fn);
    return GI_OK;
}

}  // namespace

extern "C" {

gi_status gi_fit_create(const gi_fit_desc* d, gi_stream stream, gi_fit** out) {
    NvtxRange nvtx_("gi_fit_create");
    if (!d || !out) return set_error(GI_ERR_INVALID_ARG, "gi_fit_create: NULL argument");
    *out = nullptr;
    gi_status st = check_desc(d, "gi_fit_create");
    if (st != GI_OK) return st;
    if (d->capacity < 1 || d->capacity > kMaxCapacity)
        return set_error(GI_ERR_INVALID_ARG, "gi_fit_create: capacity outside [1, 2^30)");
    const bool codec = d->codec_bits != 0;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    std::vector<ImgDesc> desc;
    int64_t tiles = 0, gauss = 0, pix = 0;
    st = image_table(d, "gi_fit_create", desc, tiles, gauss, pix);
    if (st != GI_OK) return st;

    gi_fit* f = new (std::nothrow) gi_fit();
    if (!f) return set_error(GI_ERR_NO_MEMORY, "gi_fit_create: host allocation failed");
    cudaGetDevice(&f->dev);
    f->nimg = d->n_images;
    f->N = gauss;
    f->npix = pix;
    f->capacity = d->capacity;
    f->use_graph = d->use_graph != 0;
    f->stage_events = d->stage_events != 0;
    f->B.one = desc[0];
    f->B.nimg = d->n_images;
    f->B.tile = d->tile;
    f->B.total_tiles = (int32_t)tiles;
    f->B.total_gauss = (int32_t)gauss;
    f->B.split = d->render_split;

    const int64_t N = std::max<int64_t>(1, gauss), P = std::max<int64_t>(1, pix);
    const int npx = d->tile * d->tile;
    const BinWs probe = bin_ws_layout(nullptr, N, f->capacity, (int)tiles);
    size_t sz[] = {
        up256(sizeof(ImgDesc) * d->n_images),   // 0 desc
        up256((size_t)N * 32), up256((size_t)N * 32), up256((size_t)N * 32), up256((size_t)N * 32),  // 1-4
        up256((size_t)P * 12), up256((size_t)P * 12),                                                // 5-6
        up256((size_t)N * 32),                                  // 7 rec
        up256((size_t)f->capacity * 32),                        // 8 rec_binned
        up256((size_t)tiles * npx * 12),                        // 9 dl_tiled
        up256((size_t)f->capacity * 32),                        // 10 partial
        up256((size_t)N * 16),                                  // 11 rect
        up256((size_t)N * 4),                                   // 12 cnt
        up256((size_t)(N + 1) * 8),                             // 13 pair_off
        256,                                                    // 14 k_dev, k_max
        up256((size_t)f->capacity * 4), up256((size_t)f->capacity * 4),  // 15-16 keys ids
        up256((size_t)tiles * 8),                               // 17 ranges
        up256((size_t)d->n_images * 8),                         // 18 loss
        256,                                                    // 19 step, done
        up256(probe.bytes),                                     // 20 bin ws
        d->optimizer == 1 ? up256((size_t)N * 32) : 0,          // 21 Adan n
        d->optimizer == 1 ? up256((size_t)N * 32) : 0,          // 22 Adan g_prev
        codec ? (size_t)256 : 0,                                // 23 gamma, beta + optimiser state
        codec ? up256((size_t)d->codec_stages * d->codec_size * 12) : 0,  // 24 codebooks
        codec ? up256((size_t)d->codec_stages * d->codec_size * 8) : 0,   // 25 EMA count
        codec ? up256((size_t)d->codec_stages * d->codec_size * 24) : 0,  // 26 EMA total
        codec ? up256((size_t)N * 4) : 0,                                 // 27 quantiser codes
        codec ? up256((size_t)N * d->codec_stages) : 0,                   // 28 RVQ indices
        codec ? up256((size_t)(6 + 4 * d->codec_stages * d->codec_size + 1) * 8 * reduce_blocks(N)) : 0,  // 29 partials
        codec ? up256((size_t)kCodecMaxVals * 8) + 256 : 0,               // 30 totals, ticket, out
        d->opacity_mode ? 7 * up256((size_t)N * 4) : 0,                   // 31 opacity state
        d->opacity_mode == 2 ? up256((size_t)f->capacity * 4) : 0,        // 32 per-pair opacity sums
        d->opacity_mode == 2 ? up256((size_t)P * 4) : 0,                  // 33 per-pixel walk lengths
        codec ? up256((size_t)N * 4) : 0,                                 // 34 FP16 positions
        up256((size_t)f->capacity * 4),                                   // 35 emission index per sorted pair
        up256((size_t)tiles * 8),                                         // 36 squared error per tile
        d->tile_queue ? up256((size_t)tiles * 4) + 256 : 0,               // 37 tile queue, head
    };
    size_t total = 0;
    for (size_t x : sz) total += x;
    cudaError_t e = cudaMalloc(&f->arena, total);
    if (e != cudaSuccess) {
        release(f);
        return set_error(GI_ERR_NO_MEMORY, "gi_fit_create: cudaMalloc(%zu) failed: %s", total, cudaGetErrorString(e));
    }
    char* p = static_cast<char*>(f->arena);
    auto at = [&](int i) {
        size_t off = 0;
        for (int j = 0; j < i; ++j) off += sz[j];
        return p + off;
    };
    f->d_desc = reinterpret_cast<ImgDesc*>(at(0));
    f->params = reinterpret_cast<float*>(at(1));
    f->m = reinterpret_cast<float*>(at(2));
    f->v = reinterpret_cast<float*>(at(3));
    f->grads = reinterpret_cast<float*>(at(4));
    f->targets = reinterpret_cast<float*>(at(5));
    f->out = reinterpret_cast<float*>(at(6));
    f->rec = reinterpret_cast<float4*>(at(7));
    f->rec_binned = reinterpret_cast<float4*>(at(8));
    f->dl_tiled = reinterpret_cast<float*>(at(9));
    f->partial = reinterpret_cast<float4*>(at(10));
    f->rect = reinterpret_cast<int4*>(at(11));
    f->cnt = reinterpret_cast<int32_t*>(at(12));
    f->pair_off = reinterpret_cast<int64_t*>(at(13));
    f->k_dev = reinterpret_cast<int64_t*>(at(14));
    f->k_max = f->k_dev + 1;
    f->keys = reinterpret_cast<uint32_t*>(at(15));
    f->ids = reinterpret_cast<uint32_t*>(at(16));
    f->ranges = reinterpret_cast<int2*>(at(17));
    f->emit = reinterpret_cast<uint32_t*>(at(35));
    f->loss_tile = reinterpret_cast<double*>(at(36));
    f->use_queue = d->tile_queue != 0;
    if (f->use_queue) {
        f->queue.order = reinterpret_cast<uint32_t*>(at(37));
        f->queue.head = reinterpret_cast<uint32_t*>(at(37) + up256((size_t)tiles * 4));
    }
    f->loss = reinterpret_cast<double*>(at(18));
    f->step = reinterpret_cast<int32_t*>(at(19));
    f->done = reinterpret_cast<uint32_t*>(at(19) + 16);
    f->bws = bin_ws_layout(at(20), N, f->capacity, (int)tiles);
    f->B.many = d->n_images > 1 ? f->d_desc : nullptr;

    f->adam.lr[0] = d->lr_means;
    f->adam.lr[1] = d->lr_chol;
    f->adam.lr[2] = d->lr_color;
    f->adam.beta1 = d->beta1;
    f->adam.beta2 = d->beta2;
    f->adam.eps = d->eps;
    f->adam.step = f->step;
    f->adam.done = f->done;
    f->adam.optimizer = d->optimizer;
    f->adam.beta3 = d->beta3;
    f->adam.lr_halve_every = d->lr_halve_every;
    f->adam.n = d->optimizer == 1 ? reinterpret_cast<float*>(at(21)) : nullptr;
    f->adam.g_prev = d->optimizer == 1 ? reinterpret_cast<float*>(at(22)) : nullptr;
    f->adam.param_mode = d->param_mode;
    f->B.param_mode = d->param_mode;
    f->adam.cov_mode = d->cov_mode;
    f->B.cov_mode = d->cov_mode;
    if (d->opacity_mode) {
        OpacCfg& O = f->B.opac;
        O.mode = d->opacity_mode;
        float* o = reinterpret_cast<float*>(at(31));
        const size_t st = up256((size_t)N * 4) / 4;
        O.logit = o;
        O.o = o + st;
        O.m = o + 2 * st;
        O.v = o + 3 * st;
        O.n = o + 4 * st;
        O.gp = o + 5 * st;
        O.grad = o + 6 * st;
        O.partial = d->opacity_mode == 2 ? reinterpret_cast<float*>(at(32)) : nullptr;
        O.n_last = d->opacity_mode == 2 ? reinterpret_cast<int32_t*>(at(33)) : nullptr;
    }
    std::vector<float> gb_init(30, 0.f);
    std::vector<float> cb_host;
    std::vector<double> ema_c, ema_t;
    if (codec) {
        CodecCfg& Q = f->B.codec;
        Q.bits = d->codec_bits;
        Q.stages = d->codec_stages;
        Q.size = d->codec_size;
        Q.qp = (float)((1 << d->codec_bits) - 1);
        Q.decay = d->ema_decay;
        Q.eps = d->ema_eps;
        Q.gb = reinterpret_cast<float*>(at(23));
        Q.codebooks = reinterpret_cast<float*>(at(24));
        Q.ema_count = reinterpret_cast<double*>(at(25));
        Q.ema_total = reinterpret_cast<double*>(at(26));
        Q.codes = reinterpret_cast<uchar4*>(at(27));
        Q.idx = reinterpret_cast<uint8_t*>(at(28));
        Q.part = reinterpret_cast<double*>(at(29));
        Q.tot = reinterpret_cast<double*>(at(30));
        Q.ticket = reinterpret_cast<unsigned*>(at(30) + up256((size_t)kCodecMaxVals * 8));
        Q.out = reinterpret_cast<double*>(at(30) + up256((size_t)kCodecMaxVals * 8) + 64);
        Q.means16 = reinterpret_cast<uint16_t*>(at(34));
        for (int i = 0; i < 3; ++i) {
            gb_init[i] = d->lsq_gamma[i];
            gb_init[3 + i] = d->lsq_beta[i];
        }
        const size_t ncb = (size_t)Q.stages * Q.size;
        cb_host.resize(ncb * 3);
        if (cudaMemcpy(cb_host.data(), d->codebooks, ncb * 12, cudaMemcpyDeviceToHost) != cudaSuccess) {
            release(f);
            return set_error(GI_ERR_INVALID_ARG, "gi_fit_create: codebooks is not a readable device buffer");
        }
        ema_c.assign(ncb, 1.0);  // one pseudo-count per entry, whose sum is the entry itself
        ema_t.resize(ncb * 3);
        for (size_t i = 0; i < ncb * 3; ++i) ema_t[i] = (double)cb_host[i];
    }

#define FIT_TRY(x)                                      \
    do {                                                \
        cudaError_t e_ = (x);                           \
        if (e_ != cudaSuccess) {                        \
            release(f);                                 \
            return set_cuda_error(e_, "gi_fit_create: " #x); \
        }                                               \
    } while (0)
    FIT_TRY(cudaMemsetAsync(f->arena, 0, total, s));
    FIT_TRY(cudaMemcpyAsync(f->d_desc, desc.data(), sizeof(ImgDesc) * desc.size(), cudaMemcpyHostToDevice, s));
    FIT_TRY(cudaMemcpyAsync(f->params, d->params, (size_t)gauss * 32, cudaMemcpyDeviceToDevice, s));
    FIT_TRY(cudaMemcpyAsync(f->targets, d->targets, (size_t)pix * 12, cudaMemcpyDeviceToDevice, s));
    if (d->opacity_mode && d->opacity_logits && gauss > 0)
        FIT_TRY(cudaMemcpyAsync(f->B.opac.logit, d->opacity_logits, (size_t)gauss * 4, cudaMemcpyDeviceToDevice, s));
    if (codec) {
        const CodecCfg& Q = f->B.codec;
        FIT_TRY(cudaMemcpyAsync(Q.gb, gb_init.data(), 30 * sizeof(float), cudaMemcpyHostToDevice, s));
        FIT_TRY(cudaMemcpyAsync(Q.codebooks, cb_host.data(), cb_host.size() * 4, cudaMemcpyHostToDevice, s));
        FIT_TRY(cudaMemcpyAsync(Q.ema_count, ema_c.data(), ema_c.size() * 8, cudaMemcpyHostToDevice, s));
        FIT_TRY(cudaMemcpyAsync(Q.ema_total, ema_t.data(), ema_t.size() * 8, cudaMemcpyHostToDevice, s));
    }
    FIT_TRY(cudaStreamSynchronize(s));
    FIT_TRY(cudaStreamCreateWithFlags(&f->cap_stream, cudaStreamNonBlocking));
    if (f->stage_events)
        for (cudaEvent_t& ev : f->ev) FIT_TRY(cudaEventCreate(&ev));
    f->target_src = f->targets;
    if (f->use_graph) FIT_TRY(capture_graphs(f));
#undef FIT_TRY
    *out = f;
    return GI_OK;
}

gi_status gi_fit_step(gi_fit* f, int32_t steps, gi_stream stream) {
    NvtxRange nvtx_("gi_fit_step");
    if (!f || steps < 0) return set_error(GI_ERR_INVALID_ARG, "gi_fit_step: bad argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    for (int i = 0; i < steps; ++i) {
        cudaError_t e = f->exec ? cudaGraphLaunch(f->exec, s) : enqueue_step(f, s);
        if (e != cudaSuccess) return set_cuda_error(e, "gi_fit_step");
    }
    return GI_OK;
}

gi_status gi_fit_set_target_source(gi_fit* f, const float* src, gi_stream stream) {
    NvtxRange nvtx_("gi_fit_set_target_source");
    if (!f) return set_error(GI_ERR_INVALID_ARG, "gi_fit_set_target_source: NULL fit");
    const float* use = f->targets;
    if (src) {
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, src) != cudaSuccess) {
            cudaGetLastError();
            return set_error(GI_ERR_INVALID_ARG, "gi_fit_set_target_source: pointer not known to CUDA");
        }
        if (a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
            if (!a.devicePointer || (a.type == cudaMemoryTypeDevice && a.device != f->dev))
                return set_error(GI_ERR_INVALID_ARG, "gi_fit_set_target_source: not addressable from this device");
            use = static_cast<const float*>(a.devicePointer);
        } else {
            return set_error(GI_ERR_INVALID_ARG,
                             "gi_fit_set_target_source: pageable host memory (pin or register it first)");
        }
    }
    if (use == f->target_src) return GI_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    GI_CUDA_TRY(cudaStreamSynchronize(s));
    GI_CUDA_TRY(cudaStreamSynchronize(f->cap_stream));
    f->target_src = use;
    if (f->use_graph) {
        destroy_graphs(f);
        const cudaError_t e = capture_graphs(f);
        if (e != cudaSuccess) {
            destroy_graphs(f);
            f->use_graph = false;  // eager launches from here on
            return set_cuda_error(e, "gi_fit_set_target_source: graph capture");
        }
    }
    return GI_OK;
}

gi_status gi_fit_render(gi_fit* f, gi_stream stream) {
    NvtxRange nvtx_("gi_fit_render");
    if (!f) return set_error(GI_ERR_INVALID_ARG, "gi_fit_render: NULL fit");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = f->render_exec ? cudaGraphLaunch(f->render_exec, s) : enqueue_forward(f, s, false);
    if (e != cudaSuccess) return set_cuda_error(e, "gi_fit_render");
    return GI_OK;
}

gi_status gi_fit_pointer(gi_fit* f, int32_t what, void** ptr) {
    if (!f || !ptr) return set_error(GI_ERR_INVALID_ARG, "gi_fit_pointer: NULL argument");
    switch (what) {
        case GI_FIT_PARAMS: *ptr = f->params; break;
        case GI_FIT_ADAM_M: *ptr = f->m; break;
        case GI_FIT_ADAM_V: *ptr = f->v; break;
        case GI_FIT_GRADS: *ptr = f->grads; break;
        case GI_FIT_OUT: *ptr = f->out; break;
        case GI_FIT_LOSS: *ptr = f->loss; break;
        case GI_FIT_STEP: *ptr = f->step; break;
        case GI_FIT_K: *ptr = f->k_dev; break;
        case GI_FIT_TARGET: *ptr = f->targets; break;
        case GI_FIT_ADAN_N: *ptr = f->adam.n; break;
        case GI_FIT_ADAN_GPREV: *ptr = f->adam.g_prev; break;
        case GI_FIT_CODEC_GB: *ptr = f->B.codec.gb; break;
        case GI_FIT_CODEBOOKS: *ptr = f->B.codec.codebooks; break;
        case GI_FIT_EMA_COUNT: *ptr = f->B.codec.ema_count; break;
        case GI_FIT_EMA_TOTAL: *ptr = f->B.codec.ema_total; break;
        case GI_FIT_CODES: *ptr = f->B.codec.codes; break;
        case GI_FIT_RVQ_IDX: *ptr = f->B.codec.idx; break;
        case GI_FIT_CODEC_OUT: *ptr = f->B.codec.out; break;
        case GI_FIT_OPACITY: *ptr = f->B.opac.logit; break;
        case GI_FIT_N_LAST: *ptr = f->B.opac.n_last; break;
        case GI_FIT_KEYS: *ptr = f->keys; break;
        case GI_FIT_IDS: *ptr = f->ids; break;
        case GI_FIT_RANGES: *ptr = f->ranges; break;
        case GI_FIT_PAIR_OFF: *ptr = f->pair_off; break;
        case GI_FIT_RECT: *ptr = f->rect; break;
        case GI_FIT_CNT: *ptr = f->cnt; break;
        case GI_FIT_MEANS16: *ptr = f->B.codec.means16; break;
        default: return set_error(GI_ERR_INVALID_ARG, "gi_fit_pointer: unknown field %d", what);
    }
    return GI_OK;
}

gi_status gi_fit_stage_times(gi_fit* f, float* ms) {
    if (!f || !ms) return set_error(GI_ERR_INVALID_ARG, "gi_fit_stage_times: NULL argument");
    if (!f->stage_events) return set_error(GI_ERR_INVALID_ARG, "gi_fit_stage_times: created without stage_events");
    GI_CUDA_TRY(cudaEventSynchronize(f->ev[5]));
    for (int i = 0; i < 5; ++i) GI_CUDA_TRY(cudaEventElapsedTime(&ms[i], f->ev[i], f->ev[i + 1]));
    return GI_OK;
}

gi_status gi_fit_count_pairs(const gi_fit_desc* d, gi_stream stream, int64_t* pairs) {
    NvtxRange nvtx_("gi_fit_count_pairs");
    if (!d || !pairs) return set_error(GI_ERR_INVALID_ARG, "gi_fit_count_pairs: NULL argument");
    gi_status st = check_desc(d, "gi_fit_count_pairs");
    if (st != GI_OK) return st;
    std::vector<ImgDesc> desc;
    int64_t tiles = 0, gauss = 0, pix = 0;
    st = image_table(d, "gi_fit_count_pairs", desc, tiles, gauss, pix);
    if (st != GI_OK) return st;
    *pairs = 0;
    if (gauss == 0) return GI_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool codec = d->codec_bits != 0;
    const int64_t N = gauss;
    const int64_t nblk = (N + kProjBlock - 1) / kProjBlock;
    // Scratch: image table, records, rectangles, counts, block sums; with the
    // codec, gamma and beta and the outputs the formation writes.
    const size_t sz[] = {up256(sizeof(ImgDesc) * desc.size()), up256((size_t)N * 32), up256((size_t)N * 16),
                         up256((size_t)N * 4), up256((size_t)nblk * 8), codec ? (size_t)256 : 0,
                         codec ? up256((size_t)N * 4) : 0, codec ? up256((size_t)N * d->codec_stages) : 0};
    size_t total = 0;
    for (size_t x : sz) total += x;
    void* arena = nullptr;
    cudaError_t e = cudaMalloc(&arena, total);
    if (e != cudaSuccess)
        return set_error(GI_ERR_NO_MEMORY, "gi_fit_count_pairs: cudaMalloc(%zu) failed: %s", total,
                         cudaGetErrorString(e));
    char* p = static_cast<char*>(arena);
    auto at = [&](int i) {
        size_t off = 0;
        for (int j = 0; j < i; ++j) off += sz[j];
        return p + off;
    };
    Batch B{};
    B.one = desc[0];
    B.many = d->n_images > 1 ? reinterpret_cast<ImgDesc*>(at(0)) : nullptr;
    B.nimg = d->n_images;
    B.tile = d->tile;
    B.total_tiles = (int32_t)tiles;
    B.total_gauss = (int32_t)gauss;
    B.param_mode = d->param_mode;
    B.cov_mode = d->cov_mode;
    float gb[6] = {d->lsq_gamma[0], d->lsq_gamma[1], d->lsq_gamma[2], d->lsq_beta[0], d->lsq_beta[1], d->lsq_beta[2]};
    if (codec) {
        CodecCfg& Q = B.codec;
        Q.bits = d->codec_bits;
        Q.stages = d->codec_stages;
        Q.size = d->codec_size;
        Q.qp = (float)((1 << d->codec_bits) - 1);
        Q.gb = reinterpret_cast<float*>(at(5));
        Q.codebooks = const_cast<float*>(d->codebooks);
        Q.codes = reinterpret_cast<uchar4*>(at(6));
        Q.idx = reinterpret_cast<uint8_t*>(at(7));
    }
    std::vector<int64_t> sums((size_t)nblk);
    e = cudaMemcpyAsync(at(0), desc.data(), sizeof(ImgDesc) * desc.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && codec) e = cudaMemcpyAsync(at(5), gb, sizeof(gb), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = launch_project(params_aos(d->params), B, reinterpret_cast<float4*>(at(1)), reinterpret_cast<int4*>(at(2)),
                           reinterpret_cast<int32_t*>(at(3)), reinterpret_cast<int64_t*>(at(4)), ZeroJob{}, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sums.data(), at(4), (size_t)nblk * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(arena);
    if (e != cudaSuccess) return set_cuda_error(e, "gi_fit_count_pairs");
    int64_t K = 0;
    for (int64_t v : sums) K += v;
    *pairs = K;
    return GI_OK;
}

gi_status gi_fit_destroy(gi_fit* f) {
    if (f) {
        cudaSetDevice(f->dev);
        cudaDeviceSynchronize();
        release(f);
    }
    return GI_OK;
}

}  // extern "C"
