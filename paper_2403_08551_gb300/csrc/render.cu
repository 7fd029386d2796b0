// render.cu -- forward accumulated-summation render (Sec. 3.2, Eq. 7) with
// the L2 reconstruction loss (Sec. 3.4) fused into the epilogue.
//
//   C_i = sum over the tile's list (ascending g) of c'_g exp(-sigma_g(i)),
//   sigma = 1/2 d^T Sigma^-1 d, d = (x + 0.5, y + 0.5) - mu.
//
// One CTA per tile. The tile's records are contiguous in rec_binned and are
// staged into shared memory by the TMA unit (1-D bulk copy, mbarrier
// completion). SPLIT warp groups each take a fixed contiguous share of every
// staged batch and accumulate all of the tile's pixels in FP32 registers (a
// lane owns a strip of PX pixels of one row, so per-row terms are hoisted);
// the SPLIT partial images are then summed in shared memory in a fixed order.
// Neighbouring pixels of a strip are evaluated as packed FP32 pairs
// (fma.rn.f32x2), halving the issue slots of the FP32 work.
// The result is deterministic run to run. sigma is evaluated as the sum of
// squares |M d|^2 with M the scaled inverse Cholesky factor of the record
// (sigma = 1/2 |L^-1 d|^2, Sec. 3.1 and Eq. 5), and exp(-sigma) as exp2 on
// the SFU (MUFU.EX2).
#include <algorithm>
#include <map>
#include <mutex>

#include "kernels.cuh"

namespace gi {
namespace {

// A lane owns a strip of PX pixels in each of ROWS consecutive rows: the
// x-dependent terms of sigma (dx, z1^2) are computed once per record and
// shared by the rows. A group of kStrips lanes covers the whole tile; SPLIT
// groups share the tile's list.
template <int T_, int PX_, int SPLIT_, int ROWS_>
struct RCfg {
    static constexpr int T = T_, PX = PX_, SPLIT = SPLIT_, ROWS = ROWS_;
    static constexpr int kPix = T * T;
    static constexpr int kStrips = kPix / (PX * ROWS);
    static constexpr int kStripsPerRow = T / PX;
    static constexpr int kThreads = kStrips * SPLIT;
    static constexpr int kWarps = kThreads / 32;
    static constexpr int kStage = 768;  // records per staging batch (24 KB)
    static constexpr int kStageBytes = kStage * 32;
    static constexpr int kPartBytes = SPLIT * 3 * kPix * 4;
    static constexpr int kSmem = kStageBytes > kPartBytes ? kStageBytes : kPartBytes;
    static_assert(kThreads % 32 == 0, "groups must fill warps");
    static_assert(T % ROWS == 0 && T % PX == 0, "strips must tile the tile");
};

// Shared memory of a render block: the staging buffer (reused for the
// partial images), the staging mbarrier, warp sums and the tile's target.
template <class Cfg>
struct RSmem {
    float4* srec;  // dynamic: Cfg::kSmem bytes
    uint64_t* bar;
    float* s_red;  // [32]
    float* s_tgt;  // [3 * Cfg::kPix], 16-byte aligned
};

// Renders tile t (the block's threads together). `phase` is the staging
// mbarrier's parity, carried from tile to tile by persistent blocks.
template <class Cfg>
__device__ __forceinline__ void render_tile(int t, uint32_t& phase, const RSmem<Cfg>& sm,
                                            const float4* __restrict__ rec_binned, const int2* __restrict__ ranges,
                                            const Batch& B, const float* __restrict__ target, float* __restrict__ out,
                                            float* __restrict__ dl_hwc, float* __restrict__ dl_tiled,
                                            double* __restrict__ loss_sum, double* __restrict__ loss_tile,
                                            uint32_t* status) {
    constexpr int T = Cfg::T, PX = Cfg::PX, SPLIT = Cfg::SPLIT, NT = Cfg::kThreads, NPIX = Cfg::kPix;
    float4* srec = sm.srec;
    float* spart = reinterpret_cast<float*>(sm.srec);  // reused after the last batch
    uint64_t* bar = sm.bar;
    float* s_red = sm.s_red;
    float* s_tgt = sm.s_tgt;
    __syncthreads();  // the previous tile's reads of the shared buffers are done

    const int bimg = image_of_tile(B, t);
    const ImgDesc d = img_desc(B, bimg);
    const int lt = t - d.tile_base;
    const int tx = lt % d.tw, ty = lt / d.tw;
    const int x0 = tx * T, y0 = ty * T;
    int2 rg = ranges[t];
    if (!gi_in_bounds(rg.x >= 0 && rg.y >= rg.x, status)) rg = make_int2(0, 0);
    const int L = rg.y - rg.x;

    constexpr int ROWS = Cfg::ROWS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int split = threadIdx.x / Cfg::kStrips;
    const int strip = threadIdx.x % Cfg::kStrips;
    const int row = (strip / Cfg::kStripsPerRow) * ROWS;
    const int col0 = (strip % Cfg::kStripsPerRow) * PX;
    const float py = (float)(y0 + row) + 0.5f;
    const float px0 = (float)(x0 + col0) + 0.5f;

    // The target pixels of this thread's epilogue are copied to shared memory
    // now (cp.async): their latency, long when the target is read from host
    // memory over the host link, overlaps the accumulation below.
    if (target) {
        for (int p = threadIdx.x; p < NPIX; p += NT) {
            const int x = x0 + p % T, y = y0 + p / T;
            if (x < d.W && y < d.H) {
                const float* src = target + 3 * (d.pix_base + (int64_t)y * d.W + x);
                cp_async4(&s_tgt[3 * p], src);
                cp_async4(&s_tgt[3 * p + 1], src + 1);
                cp_async4(&s_tgt[3 * p + 2], src + 2);
            }
        }
    }

    // Packed FP32 pairs: acc[r][p] holds two neighbouring pixels of row r.
    constexpr int NP2 = PX / 2;
    float2 accr[ROWS][NP2], accg[ROWS][NP2], accb[ROWS][NP2];
#pragma unroll
    for (int r = 0; r < ROWS; ++r)
#pragma unroll
        for (int p = 0; p < NP2; ++p) accr[r][p] = accg[r][p] = accb[r][p] = make_float2(0.f, 0.f);

    bool ok = true;
    for (int j0 = 0; j0 < L && ok; j0 += Cfg::kStage) {
        const int nb = min(Cfg::kStage, L - j0);
        if (threadIdx.x == 0) {
            mbar_arrive_expect_tx(bar, (uint32_t)nb * 32u);
            bulk_g2s(srec, rec_binned + 2 * ((int64_t)rg.x + j0), (uint32_t)nb * 32u, bar);
        }
        bool arrived = mbar_wait(bar, phase);
        if (!arrived) {
            // Give up on this tile after a second bounded wait for the copy.
            flag_error(status, kErrTimeout);
            mbar_wait(bar, phase);
        }
        ok = __syncthreads_and(arrived) != 0;  // block-uniform decision
        phase ^= 1u;
        const int k0 = (nb * split) / SPLIT, k1 = (nb * (split + 1)) / SPLIT;
        if (ok) {
#pragma unroll 1
            for (int k = k0; k < k1; ++k) {
                const float4 r0 = srec[2 * k];      // mx, my, m11, m21 (scaled inverse Cholesky factor)
                const float4 r1 = srec[2 * k + 1];  // m22, c'r, c'g, c'b
                const float dy = py - r0.y;
                const float dx0 = px0 - r0.x;
                const float2 M11 = make_float2(r0.z, r0.z), M21 = make_float2(r0.w, r0.w);
                float2 Z2Y[ROWS];
                const float z2y0 = r1.x * dy;
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    const float z2y = r ? fmaf(r1.x, (float)r, z2y0) : z2y0;  // m22 (dy + r)
                    Z2Y[r] = make_float2(z2y, z2y);
                }
                const float2 cr = make_float2(r1.y, r1.y), cg = make_float2(r1.z, r1.z), cb = make_float2(r1.w, r1.w);
                const float2 d0 = make_float2(dx0, dx0 + 1.0f);
#pragma unroll
                for (int p = 0; p < NP2; ++p) {
                    const float2 dx = __fadd2_rn(d0, make_float2(2.0f * p, 2.0f * p));
                    const float2 z1 = __fmul2_rn(M11, dx);
                    const float2 z1s = __fmul2_rn(z1, z1);
#pragma unroll
                    for (int r = 0; r < ROWS; ++r) {
                        const float2 z2 = __ffma2_rn(M21, dx, Z2Y[r]);
                        const float2 q = __ffma2_rn(z2, z2, z1s);            // sigma log2(e)
                        const float2 w = make_float2(ex2(-q.x), ex2(-q.y));  // exp(-sigma) of both pixels
                        accr[r][p] = __ffma2_rn(cr, w, accr[r][p]);
                        accg[r][p] = __ffma2_rn(cg, w, accg[r][p]);
                        accb[r][p] = __ffma2_rn(cb, w, accb[r][p]);
                    }
                }
            }
        }
        __syncthreads();
    }

    // Partial images of the SPLIT groups -> shared memory, [split][c][pixel].
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
#pragma unroll
        for (int q = 0; q < NP2; ++q) {
            const int p = (row + r) * T + col0 + 2 * q;
            spart[(split * 3 + 0) * NPIX + p] = accr[r][q].x;
            spart[(split * 3 + 0) * NPIX + p + 1] = accr[r][q].y;
            spart[(split * 3 + 1) * NPIX + p] = accg[r][q].x;
            spart[(split * 3 + 1) * NPIX + p + 1] = accg[r][q].y;
            spart[(split * 3 + 2) * NPIX + p] = accb[r][q].x;
            spart[(split * 3 + 2) * NPIX + p + 1] = accb[r][q].y;
        }
    }
    __syncthreads();

    const float scale = 2.0f / (3.0f * (float)d.W * (float)d.H);
    float lsum = 0.f;
    if (target) cp_async_wait_all();  // each thread reads back only the pixels it copied
    __syncthreads();                  // (the copies of a quad below may come from several threads)
    // Epilogue on quads of four neighbouring pixels of a row: 16-byte loads
    // of the partial images, the target and the planar dL/dC, and the quad's
    // twelve HWC floats as three 16-byte stores where they are aligned.
    for (int q = threadIdx.x; q < NPIX / 4; q += NT) {
        const int p = 4 * q;
        float4 C[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float4 sacc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int sp = 0; sp < SPLIT; ++sp) {
                const float4 u = *reinterpret_cast<const float4*>(&spart[(sp * 3 + c) * NPIX + p]);
                sacc.x += u.x;
                sacc.y += u.y;
                sacc.z += u.z;
                sacc.w += u.w;
            }
            C[c] = sacc;
        }
        // HWC order of the quad: r0 g0 b0 r1 g1 b1 r2 g2 b2 r3 g3 b3
        float hwc[12] = {C[0].x, C[1].x, C[2].x, C[0].y, C[1].y, C[2].y,
                         C[0].z, C[1].z, C[2].z, C[0].w, C[1].w, C[2].w};
        const int x = x0 + p % T, y = y0 + p / T;
        const int nx = y < d.H ? max(0, min(4, d.W - x)) : 0;  // pixels of the quad inside the image
        float dl[12];
#pragma unroll
        for (int i = 0; i < 12; ++i) dl[i] = 0.f;
        if (target && nx > 0) {
            float tg[12];
            const float4* tq = reinterpret_cast<const float4*>(&s_tgt[3 * p]);
            *reinterpret_cast<float4*>(&tg[0]) = tq[0];
            *reinterpret_cast<float4*>(&tg[4]) = tq[1];
            *reinterpret_cast<float4*>(&tg[8]) = tq[2];
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                if (i < 3 * nx) {
                    const float r = hwc[i] - tg[i];
                    lsum = fmaf(r, r, lsum);
                    dl[i] = r * scale;
                }
            }
        }
        if (nx > 0) {
            const int64_t pix = d.pix_base + (int64_t)y * d.W + x;
            float* o = out + 3 * pix;
            if (nx == 4 && (reinterpret_cast<uintptr_t>(o) & 15) == 0) {
                float4* o4 = reinterpret_cast<float4*>(o);
                o4[0] = make_float4(hwc[0], hwc[1], hwc[2], hwc[3]);
                o4[1] = make_float4(hwc[4], hwc[5], hwc[6], hwc[7]);
                o4[2] = make_float4(hwc[8], hwc[9], hwc[10], hwc[11]);
            } else {
#pragma unroll
                for (int i = 0; i < 12; ++i)
                    if (i < 3 * nx) o[i] = hwc[i];
            }
            if (target && dl_hwc) {
                float* dh = dl_hwc + 3 * pix;
#pragma unroll
                for (int i = 0; i < 12; ++i)
                    if (i < 3 * nx) dh[i] = dl[i];
            }
        }
        if (dl_tiled) {  // planar per tile: R, G, B planes of T*T floats
            float4* dt = reinterpret_cast<float4*>(dl_tiled + (int64_t)t * 3 * NPIX);
            dt[q] = make_float4(dl[0], dl[3], dl[6], dl[9]);
            dt[NPIX / 4 + q] = make_float4(dl[1], dl[4], dl[7], dl[10]);
            dt[2 * NPIX / 4 + q] = make_float4(dl[2], dl[5], dl[8], dl[11]);
        }
    }
    if (target && (loss_sum || loss_tile)) {
        // fixed order: butterfly within warps, then the warps in order
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
        if (lane == 0) s_red[warp] = lsum;
        __syncthreads();
        if (threadIdx.x == 0) {
            float s = 0.f;
            for (int w = 0; w < Cfg::kWarps; ++w) s += s_red[w];
            if (loss_tile) loss_tile[t] = (double)s;
            else atomicAdd(&loss_sum[bimg], (double)s);
        }
    }
}

// One block per tile, tiles in index order.
template <class Cfg>
__global__ void __launch_bounds__(Cfg::kThreads) k_render(const float4* __restrict__ rec_binned,
                                                          const int2* __restrict__ ranges, Batch B,
                                                          const float* __restrict__ target, float* __restrict__ out,
                                                          float* __restrict__ dl_hwc, float* __restrict__ dl_tiled,
                                                          double* __restrict__ loss_sum, double* __restrict__ loss_tile,
                                                          uint32_t* status) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ float s_red[32];
    __shared__ __align__(16) float s_tgt[3 * Cfg::kPix];
    const RSmem<Cfg> sm{reinterpret_cast<float4*>(smem), &bar, s_red, s_tgt};
    pdl_wait();
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    uint32_t phase = 0;
    render_tile<Cfg>(blockIdx.x, phase, sm, rec_binned, ranges, B, target, out, dl_hwc, dl_tiled, loss_sum, loss_tile,
                     status);
}

// Persistent blocks (one wave) pulling tiles from the queue: queue.order
// holds the tiles by descending list length, queue.head counts the tiles
// handed out (zero at launch). A block asks for its next tile as it starts
// the current one, so the atomic's latency is hidden. Each tile's result is
// the same whichever block renders it and when.
template <class Cfg>
__global__ void __launch_bounds__(Cfg::kThreads) k_render_queued(const float4* __restrict__ rec_binned,
                                                                 const int2* __restrict__ ranges, Batch B,
                                                                 const float* __restrict__ target,
                                                                 float* __restrict__ out, float* __restrict__ dl_hwc,
                                                                 float* __restrict__ dl_tiled,
                                                                 double* __restrict__ loss_sum,
                                                                 double* __restrict__ loss_tile, TileQueue queue,
                                                                 uint32_t* status) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ float s_red[32];
    __shared__ __align__(16) float s_tgt[3 * Cfg::kPix];
    __shared__ uint32_t s_next;
    const RSmem<Cfg> sm{reinterpret_cast<float4*>(smem), &bar, s_red, s_tgt};
    pdl_wait();
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        s_next = atomicAdd(queue.head, 1u);
    }
    __syncthreads();
    uint32_t phase = 0;
    const uint32_t ntiles = (uint32_t)B.total_tiles;
    uint32_t idx = s_next;
    while (idx < ntiles) {
        uint32_t nxt = 0;
        if (threadIdx.x == 0) nxt = atomicAdd(queue.head, 1u);  // read back after the tile
        const uint32_t t = queue.order[idx];
        if (gi_in_bounds(t < ntiles, status))
            render_tile<Cfg>((int)t, phase, sm, rec_binned, ranges, B, target, out, dl_hwc, dl_tiled, loss_sum,
                             loss_tile, status);
        __syncthreads();
        if (threadIdx.x == 0) s_next = nxt;
        __syncthreads();
        idx = s_next;
    }
}

// The tile queue: tiles ordered by descending list length (lengths above
// kQueueBuckets - 1 share the first bucket; inside a bucket the order is
// whatever the atomics give, which no result depends on), and the head
// counter reset. One block.
constexpr int kQueueBuckets = 4096;
constexpr int kQueueThreads = 1024;

__global__ void __launch_bounds__(kQueueThreads) k_tile_queue(const int2* __restrict__ ranges, int total_tiles,
                                                              TileQueue queue) {
    __shared__ uint32_t s_cnt[kQueueBuckets];
    __shared__ uint32_t s_warp[32];
    pdl_wait();
    for (int i = threadIdx.x; i < kQueueBuckets; i += blockDim.x) s_cnt[i] = 0u;
    __syncthreads();
    auto bucket = [&](int t) {
        const int2 rg = ranges[t];
        const int L = max(0, rg.y - rg.x);
        return kQueueBuckets - 1 - min(L, kQueueBuckets - 1);  // longest first
    };
    for (int t = threadIdx.x; t < total_tiles; t += blockDim.x) atomicAdd(&s_cnt[bucket(t)], 1u);
    __syncthreads();
    // exclusive scan of the bucket counts, four buckets per thread
    constexpr int PER = kQueueBuckets / kQueueThreads;
    uint32_t v[PER], sum = 0;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        v[i] = s_cnt[threadIdx.x * PER + i];
        sum += v[i];
    }
    const uint32_t incl = block_incl_scan<uint32_t>(sum, s_warp);
    uint32_t run = incl - sum;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        s_cnt[threadIdx.x * PER + i] = run;
        run += v[i];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < total_tiles; t += blockDim.x) queue.order[atomicAdd(&s_cnt[bucket(t)], 1u)] = t;
    if (threadIdx.x == 0) *queue.head = 0u;
}

template <class Cfg>
int render_blocks_per_sm() {
    static std::mutex mu;
    static std::map<int, int> cached;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    std::lock_guard<std::mutex> lk(mu);
    int& v = cached[dev];
    if (v <= 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_queued<Cfg>, Cfg::kThreads, Cfg::kSmem) !=
                cudaSuccess ||
            nb <= 0)
            nb = 1;
        v = nb;
    }
    return v;
}

template <class Cfg>
cudaError_t launch_cfg(const float4* rec_binned, const int2* ranges, const Batch& B, const float* target,
                       float* out, float* dl_hwc, float* dl_tiled, double* loss_sum, double* loss_tile,
                       const TileQueue* queue, uint32_t* status, cudaStream_t s) {
    static_assert(Cfg::kSmem <= 96 * 1024, "dynamic shared memory of the render");
    if (B.total_tiles <= 0) return cudaSuccess;
    // the dynamic window plus the static part may exceed the default 48 KB
    if (queue) {
        cudaError_t e = smem_optin(reinterpret_cast<const void*>(k_render_queued<Cfg>), Cfg::kSmem);
        if (e != cudaSuccess) return e;
        e = launch_pdl(k_tile_queue, dim3(1), dim3(kQueueThreads), 0, s, ranges, B.total_tiles, *queue);
        if (e != cudaSuccess) return e;
        const int blocks = std::max(1, std::min(B.total_tiles, sm_count() * render_blocks_per_sm<Cfg>()));
        return launch_pdl(k_render_queued<Cfg>, dim3(blocks), dim3(Cfg::kThreads), Cfg::kSmem, s, rec_binned, ranges,
                          B, target, out, dl_hwc, dl_tiled, loss_sum, loss_tile, *queue, status);
    }
    const cudaError_t e = smem_optin(reinterpret_cast<const void*>(k_render<Cfg>), Cfg::kSmem);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_render<Cfg>, dim3(B.total_tiles), dim3(Cfg::kThreads), Cfg::kSmem, s, rec_binned, ranges, B,
                      target, out, dl_hwc, dl_tiled, loss_sum, loss_tile, status);
}

}  // namespace

cudaError_t launch_render(const float4* rec_binned, const int2* ranges, const Batch& B, const float* target,
                          float* out, float* dl_hwc, float* dl_tiled, double* loss_sum, double* loss_tile,
                          uint32_t* status, cudaStream_t s, const TileQueue* queue) {
    // split: lane groups that share one tile's list (each group covers all
    // of the tile's pixels); 0 picks the default for the tile edge. Tile 16
    // gives a lane a block 4 pixels wide (the rows share each column's
    // terms): 4 rows (16 lanes per group) with split 4, 8 rows (8 lanes per
    // group, 64 threads per block) with split 8; tiles 8 and 32 a strip of
    // one row.
    const int sp = B.split;
    switch (B.tile) {
        case 8:
            if (sp == 2)
                return launch_cfg<RCfg<8, 2, 2, 1>>(rec_binned, ranges, B, target, out, dl_hwc, dl_tiled, loss_sum,
                                                    loss_tile, queue, status, s);
            if (sp == 0 || sp == 4)
                return launch_cfg<RCfg<8, 2, 4, 1>>(rec_binned, ranges, B, target, out, dl_hwc, dl_tiled, loss_sum,
                                                    loss_tile, queue, status, s);
            return cudaErrorInvalidValue;
        case 16:
            if (sp == 4)
                return launch_cfg<RCfg<16, 4, 4, 4>>(rec_binned, ranges, B, target, out, dl_hwc, dl_tiled, loss_sum,
                                                     loss_tile, queue, status, s);
            if (sp == 0 || sp == 8)
                return launch_cfg<RCfg<16, 4, 8, 8>>(rec_binned, ranges, B, target, out, dl_hwc, dl_tiled, loss_sum,
                                                     loss_tile, queue, status, s);
            return cudaErrorInvalidValue;
        case 32:
            if (sp == 1)
                return launch_cfg<RCfg<32, 8, 1, 1>>(rec_binned, ranges, B, target, out, dl_hwc, dl_tiled, loss_sum,
                                                     loss_tile, queue, status, s);
            if (sp == 0 || sp == 2)
                return launch_cfg<RCfg<32, 8, 2, 1>>(rec_binned, ranges, B, target, out, dl_hwc, dl_tiled, loss_sum,
                                                     loss_tile, queue, status, s);
            return cudaErrorInvalidValue;
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace gi
