// backward.cu -- gradients of the accumulated-summation render (App. A).
//
// Pass 1 (k_backward): a lane owns one (tile, Gaussian) pair at a time. It
// walks every pixel of the tile, recomputing
// w = exp(-sigma) (no per-pixel state is kept from the forward pass) and
// accumulates eight sums per pair:
//   gc      = sum_i G_i w_i                        -> dL/dc'       (App. A.1)
//   e~_i    = <G_i, c'> w_i  (dL/dsigma_i = -e~_i; App. A.1 writes
//             dC/dsigma = -exp(-sigma) without the factor c', restored here)
//   S_x, S_y, S_xx, S_xy, S_yy = sum_i e~_i (dx, dy, dx^2, dx dy, dy^2)
// with d = p - mu. Warps never reduce across lanes and there are no atomics:
// the eight sums are stored at the pair's emission index pair_off[g] + j,
// so pass 2 can reduce them per Gaussian in a fixed order (deterministic).
//
// Pass 2 (k_reduce): per Gaussian, sum its pairs in emission order, then
//   dL/dA = -S_xx/2, dL/dB = -S_xy, dL/dC = -S_yy/2   (Sigma^-1 = [[A,B],[B,C]])
//   dL/dmu = (A S_x + B S_y, B S_x + C S_y)           (dsigma/dmu = -Sigma^-1 d)
//   dL/dSigma = -Q G_Q Q, G_Q = [[dL/dA, dL/dB/2], [dL/dB/2, dL/dC]]
//   dL/dl1 = 2 g1 l1 + 2 g2 l2, dL/dl2 = 2 g2 l1 + 2 g3 l2, dL/dl3 = 2 g3 l3
// (App. A.2 with G = dL/dSigma = [[g1, g2], [g2, g3]]; the printed dL/dl2
// has "g2 l2" where Sigma22 = l2^2 + l3^2 gives 2 g3 l2.) Optionally followed
// by an Adam step (Kingma & Ba, bias-corrected) on the AoS parameters.
#include <algorithm>
#include <map>
#include <mutex>

#include "kernels.cuh"

namespace gi {
namespace {

// s + x with the lost low-order part carried in c (Kahan); explicit
// round-to-nearest operations so the compensation is not contracted away.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// Sums of one row of the tile for one pair: u = sum e, v = sum e dx,
// qm = sum e dx^2 over the row's pixels (e = <G, c'> w) and the colour sums
// gc += G w. dL/dC is planar per tile (R, G, B planes of T*T floats), so one
// float4 load gives four neighbouring pixels of a channel, and the arithmetic
// runs on packed FP32 pairs (fma/add/mul.rn.f32x2): each instruction
// advances two pixels. dx, dx^2 and z1^2 = (m11 dx)^2 of the row's pixel
// pairs do not depend on the row and are passed in registers for tiles of up
// to 16 x 16, so a pixel pair costs two packed operations for sigma.
template <int T, bool kHoist, int NH>
__device__ __forceinline__ void row_sums(const float* __restrict__ G, int y, float2 M11, float2 M21, float z2y,
                                         float2 cr, float2 cg, float2 cb, float2 d0, const float2 (&DX)[NH],
                                         const float2 (&DX2)[NH], const float2 (&Z1S)[NH], float2& gcr, float2& gcg,
                                         float2& gcb, float& us, float& vs, float& qs) {
    constexpr int NPIX = T * T;
    const float2 Z2Y = make_float2(z2y, z2y);
    float2 u = make_float2(0.f, 0.f), v = u, qm = u;
    const float4* Rr = reinterpret_cast<const float4*>(G + y * T);
    const float4* Rg = reinterpret_cast<const float4*>(G + NPIX + y * T);
    const float4* Bb_ = reinterpret_cast<const float4*>(G + 2 * NPIX + y * T);
#pragma unroll
    for (int x4 = 0; x4 < T / 4; ++x4) {
        const float4 R = Rr[x4], Gg = Rg[x4], Bb = Bb_[x4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float2 gr = h ? make_float2(R.z, R.w) : make_float2(R.x, R.y);
            const float2 gg = h ? make_float2(Gg.z, Gg.w) : make_float2(Gg.x, Gg.y);
            const float2 gb = h ? make_float2(Bb.z, Bb.w) : make_float2(Bb.x, Bb.y);
            const float xo = (float)(4 * x4 + 2 * h);
            const int hi = kHoist ? 2 * x4 + h : 0;
            const float2 dx = kHoist ? DX[hi] : __fadd2_rn(d0, make_float2(xo, xo));
            const float2 z2 = __ffma2_rn(M21, dx, Z2Y);
            float2 z1s;
            if (kHoist) {
                z1s = Z1S[hi];
            } else {
                const float2 z1 = __fmul2_rn(M11, dx);
                z1s = __fmul2_rn(z1, z1);
            }
            const float2 q = __ffma2_rn(z2, z2, z1s);            // sigma log2(e) = |M d|^2
            const float2 w = make_float2(ex2(-q.x), ex2(-q.y));  // exp(-sigma)
            gcr = __ffma2_rn(gr, w, gcr);
            gcg = __ffma2_rn(gg, w, gcg);
            gcb = __ffma2_rn(gb, w, gcb);
            const float2 gw = __ffma2_rn(gb, cb, __ffma2_rn(gg, cg, __fmul2_rn(gr, cr)));
            const float2 e = __fmul2_rn(gw, w);
            u = __fadd2_rn(u, e);
            if (kHoist) {
                v = __ffma2_rn(e, dx, v);
                qm = __ffma2_rn(e, DX2[hi], qm);
            } else {
                const float2 t1 = __fmul2_rn(e, dx);
                v = __fadd2_rn(v, t1);
                qm = __ffma2_rn(t1, dx, qm);
            }
        }
    }
    us = u.x + u.y;
    vs = v.x + v.y;
    qs = qm.x + qm.y;
}

// Walks the T x T pixels of one tile for one pair and returns its eight
// sums. The moment sums are Kahan-compensated across pairs of rows: the
// per-pair sums cancel strongly for Gaussians near equilibrium, and the row
// partials are the large terms of that cancellation.
template <int T>
__device__ __forceinline__ void pair_sums(const float* __restrict__ G, float4 r0, float4 r1, float dx0, float dyb,
                                          float (&out)[8]) {
    const float2 M11 = make_float2(r0.z, r0.z), M21 = make_float2(r0.w, r0.w);
    const float2 cr = make_float2(r1.y, r1.y), cg = make_float2(r1.z, r1.z), cb = make_float2(r1.w, r1.w);
    const float2 d0 = make_float2(dx0, dx0 + 1.0f);
    constexpr bool kHoist = T <= 16;
    constexpr int NH = kHoist ? T / 2 : 1;
    float2 DX[NH], DX2[NH], Z1S[NH];
    if (kHoist) {
#pragma unroll
        for (int i = 0; i < NH; ++i) {
            DX[i] = __fadd2_rn(d0, make_float2(2.0f * i, 2.0f * i));
            DX2[i] = __fmul2_rn(DX[i], DX[i]);
            const float2 z1 = __fmul2_rn(M11, DX[i]);
            Z1S[i] = __fmul2_rn(z1, z1);
        }
    }
    float2 gcr = make_float2(0.f, 0.f), gcg = gcr, gcb = gcr;
    float S[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, cS[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
    for (int y = 0; y < T; y += 2) {
        const float dy0 = dyb + (float)y, dy1 = dy0 + 1.0f;
        float us0, vs0, qs0, us1, vs1, qs1;
        row_sums<T, kHoist, NH>(G, y, M11, M21, r1.x * dy0, cr, cg, cb, d0, DX, DX2, Z1S, gcr, gcg, gcb, us0, vs0,
                                qs0);
        row_sums<T, kHoist, NH>(G, y + 1, M11, M21, r1.x * dy1, cr, cg, cb, d0, DX, DX2, Z1S, gcr, gcg, gcb, us1,
                                vs1, qs1);
        const float a0 = us0 * dy0, a1 = us1 * dy1;
        kahan_add(S[0], cS[0], vs0 + vs1);
        kahan_add(S[1], cS[1], a0 + a1);
        kahan_add(S[2], cS[2], qs0 + qs1);
        kahan_add(S[3], cS[3], vs0 * dy0 + vs1 * dy1);
        kahan_add(S[4], cS[4], a0 * dy0 + a1 * dy1);
    }
    out[0] = gcr.x + gcr.y;
    out[1] = gcg.x + gcg.y;
    out[2] = gcb.x + gcb.y;
#pragma unroll
    for (int m = 0; m < 5; ++m) out[3 + m] = S[m] - cS[m];
}

__device__ __forceinline__ void tile_origin(const Batch& B, uint32_t t, int T, int& tx, int& ty) {
    const ImgDesc d = img_desc(B, image_of_tile(B, (int)t));
    const int lt = (int)t - d.tile_base;
    tx = lt % d.tw;
    ty = lt / d.tw;
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

constexpr int kBwdWarps = 8;  // warps per backward block
constexpr int kBwdThreads = kBwdWarps * 32;

// Planar dL/dC floats of one tile.
template <int T>
__host__ __device__ constexpr int tile_floats() { return 3 * T * T; }
// Tiles of up to 16 x 16 pixels are staged in shared memory, two slots per warp.
template <int T>
__host__ __device__ constexpr bool stage_dl() { return T <= 16; }

// Shared memory of one warp: the records, tile keys and emission indices of
// its current and next task (double buffer), then the two staged tiles.
template <int T>
struct BwdWarpSmem {
    float4 rec[2][64];
    uint32_t key[2][32];
    uint32_t emit[2][32];
    float g[stage_dl<T>() ? 2 * tile_floats<T>() : 4];
};
template <int T>
constexpr size_t backward_smem() { return kBwdWarps * sizeof(BwdWarpSmem<T>); }

// cp.async of the records, keys and emission indices of the 32 pairs of
// task `task` (pairs 32 task .. 32 task + 31, those below K) into buffer b.
template <int T>
__device__ __forceinline__ void prefetch_task(BwdWarpSmem<T>& w, int b, int task, int K, int lane,
                                              const float4* __restrict__ rec_binned, const uint32_t* __restrict__ keys,
                                              const uint32_t* __restrict__ emit) {
    const int k0 = task * 32;
#pragma unroll
    for (int c = lane; c < 64; c += 32)  // 16-byte halves of the 32-byte records
        if (k0 + (c >> 1) < K) cp_async16(&w.rec[b][c], rec_binned + 2 * (size_t)k0 + c);
    if (lane < 16) {  // lanes 0-7: keys, 8-15: emission indices, four per copy
        const int c = lane & 7;
        const uint32_t* src = (lane < 8 ? keys : emit) + k0 + 4 * c;
        uint32_t* dst = (lane < 8 ? w.key[b] : w.emit[b]) + 4 * c;
        if (k0 + 4 * c + 3 < K) {
            cp_async16(dst, src);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (k0 + 4 * c + e < K) cp_async4(dst + e, src + e);
        }
    }
}

// Persistent backward: one warp task = 32 consecutive pairs of the sorted
// list, one per lane (uniform work: every pair walks T x T pixels). Warp r
// of the grid (ranked block-minor, so that the warps with one task more are
// spread over all SMs) owns a contiguous range of tasks; while it works on
// one task, the records, keys and emission indices of the next are already
// on their way to its shared memory (cp.async, double-buffered), so the
// warps of an SM, which run equal-length tasks in step, do not all wait on
// global memory at the same time. Tiles of up to 16 x 16: the warp keeps
// two tiles of planar dL/dC in shared memory and reloads a slot only when
// a task needs a tile it does not hold (consecutive tasks mostly share
// tiles); a task whose pairs span more than two tiles (tiles with fewer than
// 32 pairs) takes one more round per extra pair of tiles. Larger tiles read
// dL/dC from global memory. Each pair's sums land at its emission index.
template <int T>
__global__ void __launch_bounds__(kBwdThreads, 2) k_backward(
    const float4* __restrict__ rec_binned, const uint32_t* __restrict__ keys, const uint32_t* __restrict__ emit,
    const float* __restrict__ dl_tiled, Batch B, const int64_t* __restrict__ k_dev, int64_t capacity,
    float4* __restrict__ partial, uint32_t* __restrict__ status) {
    constexpr int TF = tile_floats<T>();
    extern __shared__ float4 s_dyn[];
    pdl_wait();
    const int K = (int)min(*k_dev, capacity);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    BwdWarpSmem<T>& w = reinterpret_cast<BwdWarpSmem<T>*>(s_dyn)[wib];
    const int nt = (K + 31) >> 5;
    const int W = gridDim.x * kBwdWarps;
    const int r = wib * gridDim.x + blockIdx.x;
    const int Q = nt / W, R = nt % W;
    const int t_begin = r * Q + min(r, R), t_end = t_begin + Q + (r < R ? 1 : 0);
    if (t_begin >= t_end) return;
    uint32_t tag[2] = {0xffffffffu, 0xffffffffu};  // tiles held by the two slots (warp-uniform)
    prefetch_task<T>(w, 0, t_begin, K, lane, rec_binned, keys, emit);
    cp_async_commit();
    int cur = 0;
    for (int task = t_begin; task < t_end; ++task, cur ^= 1) {
        cp_async_wait<0>();  // this task's records
        __syncwarp();
        const int k = task * 32 + lane;
        const bool valid = k < K;
        const float4 r0 = w.rec[cur][2 * lane], r1 = w.rec[cur][2 * lane + 1];
        uint32_t t = w.key[cur][lane];
        const uint32_t p = w.emit[cur][lane];
        const bool inb = gi_in_bounds(!valid || t < (uint32_t)B.total_tiles, status);
        if (!inb) t = 0;
        int tx = 0, ty = 0;
        if (valid) tile_origin(B, t, T, tx, ty);
        const float dx0 = (float)(tx * T) + 0.5f - r0.x, dyb = (float)(ty * T) + 0.5f - r0.y;
        float o[8];
        bool have = false;
        uint32_t pending = __ballot_sync(0xffffffffu, valid && inb);
        bool first = true;
        do {
            if (stage_dl<T>()) {
                // Tiles of the first and last pending lanes; slots reloaded
                // only for tiles the warp does not hold.
                const uint32_t ta = __shfl_sync(0xffffffffu, t, __ffs(pending) - 1);
                const uint32_t tb = __shfl_sync(0xffffffffu, t, 31 - __clz(pending));
                const bool ha = tag[0] == ta || tag[1] == ta, hb = tag[0] == tb || tag[1] == tb;
                if (!ha || !hb) {
                    // keep the slot that holds a needed tile, fill the other(s)
                    int keep = -1;
                    if (tag[0] == ta || tag[0] == tb) keep = 0;
                    else if (tag[1] == ta || tag[1] == tb) keep = 1;
                    const uint32_t need0 = ha ? tb : ta;  // the first missing tile
                    const int s0 = keep == 0 ? 1 : 0;
                    const float4* src0 = reinterpret_cast<const float4*>(dl_tiled + (size_t)need0 * TF);
                    float4* dst0 = reinterpret_cast<float4*>(w.g + s0 * TF);
                    for (int i = lane; i < TF / 4; i += 32) cp_async16(dst0 + i, src0 + i);
                    tag[s0] = need0;
                    if (!ha && !hb && tb != ta) {  // both missing: the second into the other slot
                        const float4* src1 = reinterpret_cast<const float4*>(dl_tiled + (size_t)tb * TF);
                        float4* dst1 = reinterpret_cast<float4*>(w.g + (1 - s0) * TF);
                        for (int i = lane; i < TF / 4; i += 32) cp_async16(dst1 + i, src1 + i);
                        tag[1 - s0] = tb;
                    }
                }
                cp_async_commit();
                if (first) {
                    // the next task's records go out behind this task's tiles
                    if (task + 1 < t_end) prefetch_task<T>(w, cur ^ 1, task + 1, K, lane, rec_binned, keys, emit);
                    cp_async_commit();
                    cp_async_wait<1>();  // the tiles (all but the newest group)
                } else {
                    cp_async_wait<0>();
                }
                __syncwarp();
                const bool mine = ((pending >> lane) & 1u) && (t == tag[0] || t == tag[1]);
                if (mine) {
                    pair_sums<T>(w.g + (t == tag[0] ? 0 : TF), r0, r1, dx0, dyb, o);
                    have = true;
                }
                pending &= ~__ballot_sync(0xffffffffu, mine);
                __syncwarp();
            } else {
                if (first && task + 1 < t_end) prefetch_task<T>(w, cur ^ 1, task + 1, K, lane, rec_binned, keys, emit);
                cp_async_commit();
                if ((pending >> lane) & 1u) {
                    pair_sums<T>(dl_tiled + (size_t)t * TF, r0, r1, dx0, dyb, o);
                    have = true;
                }
                pending = 0;
            }
            first = false;
        } while (pending);
        if (have) {
            if (p < (uint64_t)capacity) {
                st_global_v8(partial + 2 * (size_t)p, make_float4(o[0], o[1], o[2], o[3]),
                             make_float4(o[4], o[5], o[6], o[7]));
            } else {
                flag_error(status, kErrBounds);
            }
        }
    }
    cp_async_wait<0>();
}

// Emission index of each sorted pair (for a binning that did not write it):
// pair_off[g] + the row-major position of its tile in g's rectangle.
__global__ void k_emit_index(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ ids,
                             const int4* __restrict__ rect, const int64_t* __restrict__ pair_off, Batch B,
                             const int64_t* __restrict__ k_dev, int64_t capacity, uint32_t* __restrict__ emit,
                             uint32_t* __restrict__ status) {
    pdl_wait();
    const int K = (int)min(*k_dev, capacity);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
        const uint32_t t = keys[k], g = ids[k];
        uint32_t e = 0xffffffffu;
        if (t < (uint32_t)B.total_tiles && g < (uint32_t)B.total_gauss) {
            const ImgDesc d = img_desc(B, image_of_tile(B, (int)t));
            const int lt = (int)t - d.tile_base;
            const int4 r = rect[g];
            e = (uint32_t)(pair_off[g] + (int64_t)(lt / d.tw - r.y) * (r.z - r.x) + (lt % d.tw - r.x));
        } else {
            flag_error(status, kErrBounds);
        }
        emit[k] = e;
    }
}

// HWC dL/dC -> planar per-tile layout (R, G, B planes), zero outside the image.
template <int T>
__global__ void k_pack_dl(const float* __restrict__ dl, Batch B, float* __restrict__ out) {
    constexpr int NPIX = T * T;
    pdl_wait();
    const int t = blockIdx.x;
    const ImgDesc d = img_desc(B, image_of_tile(B, t));
    const int lt = t - d.tile_base;
    const int tx = lt % d.tw, ty = lt / d.tw;
    for (int p = threadIdx.x; p < NPIX; p += blockDim.x) {
        const int x = tx * T + p % T, y = ty * T + p / T;
        float r = 0.f, g = 0.f, bl = 0.f;
        if (x < d.W && y < d.H) {
            const int64_t pix = d.pix_base + (int64_t)y * d.W + x;
            r = dl[3 * pix];
            g = dl[3 * pix + 1];
            bl = dl[3 * pix + 2];
        }
        float* o = out + (size_t)t * 3 * NPIX;
        o[p] = r;
        o[NPIX + p] = g;
        o[2 * NPIX + p] = bl;
    }
}

constexpr int kReduceThreads = 128;
constexpr int kReduceRows = 128;  // pair rows a warp stages per chunk

// Codec sums, stage 1 (Sec. 3.3-3.4): per block, dL/dgamma, dL/dbeta, the
// commitment term and, per RVQ stage and codebook entry, the count and the
// residual sum of the Gaussians assigned to it. Warp sums by butterfly, then
// the block's warps in order: a fixed summation order, so the totals do not
// depend on scheduling. Row v of Q.part holds value v of each of the nb
// Gaussian blocks; this block is number blk of them.
__device__ void codec_block_partials(const CodecCfg& Q, const float (&gb)[6], const int (&jj)[kCodecMaxStages],
                                     const float (&rr)[kCodecMaxStages][3], float commit, int blk, int nb) {
    constexpr int kWarps = kReduceThreads / 32;
    extern __shared__ float s_cv_dyn[];  // [kWarps][nv] (dynamic: sized by the codebooks)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nv = codec_nvals(Q);
    float* s_cv = s_cv_dyn + warp * nv;
#pragma unroll
    for (int v = 0; v < 6; ++v) {
        const float w = warp_sum(gb[v]);
        if (lane == 0) s_cv[v] = w;
    }
    {
        const float w = warp_sum(commit);
        if (lane == 0) s_cv[nv - 1] = w;
    }
#pragma unroll
    for (int m = 0; m < kCodecMaxStages; ++m) {
        if (m < Q.stages) {
            for (int j = 0; j < Q.size; ++j) {
                const bool mine = jj[m] == j;
                const unsigned mask = __ballot_sync(0xffffffffu, mine);
                float c0 = 0.f, c1 = 0.f, c2 = 0.f;
                if (mask) {  // warp-uniform
                    c0 = warp_sum(mine ? rr[m][0] : 0.f);
                    c1 = warp_sum(mine ? rr[m][1] : 0.f);
                    c2 = warp_sum(mine ? rr[m][2] : 0.f);
                }
                if (lane == 0) {
                    float* o = &s_cv[6 + (m * Q.size + j) * 4];
                    o[0] = (float)__popc(mask);
                    o[1] = c0;
                    o[2] = c1;
                    o[3] = c2;
                }
            }
        }
    }
    __syncthreads();
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
        double acc = 0.0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) acc += (double)s_cv_dyn[w * nv + v];
        Q.part[(size_t)v * nb + blk] = acc;
    }
}

// The optimiser step of one scalar parameter (Adam, or Adan without weight
// decay), with the block's bias corrections s_bc and step count.
__device__ __forceinline__ float opt_step(const AdamCfg& cfg, const float* s_bc, int step, float lr, float gr, float p,
                                          float& m, float& v, float* n, float* gp) {
    if (cfg.optimizer == 1) {
        const float dg = step == 1 ? 0.f : gr - *gp;
        m = cfg.beta1 * m + (1.f - cfg.beta1) * gr;
        v = cfg.beta2 * v + (1.f - cfg.beta2) * dg;
        const float ge = gr + cfg.beta2 * dg;
        *n = cfg.beta3 * *n + (1.f - cfg.beta3) * ge * ge;
        *gp = gr;
        return p - lr * (m * s_bc[0] + cfg.beta2 * (v * s_bc[1])) / (sqrtf(*n) * s_bc[2] + cfg.eps);
    }
    m = cfg.beta1 * m + (1.f - cfg.beta1) * gr;
    v = cfg.beta2 * v + (1.f - cfg.beta2) * gr * gr;
    return p - (lr * s_bc[0]) * m / (sqrtf(v) * s_bc[1] + cfg.eps);
}

// One thread per Gaussian. A warp's 32 Gaussians own one contiguous range of
// pair rows, which the warp stages through shared memory in chunks of
// coalesced cp.async copies, the next chunk in flight while one is summed;
// per slot each Gaussian's rows are summed in emission order, Kahan-
// compensated. Then the conic and Cholesky chain (App. A.2), the chains of
// the parameterisation, covariance form, codec and opacity modes, and the
// optimiser step. With loss_tile, one block per image precedes the
// Gaussians' blocks and sums that image's squared error.
template <bool ADAM, bool CODEC = false, int OPAC = 0>
__global__ void __launch_bounds__(kReduceThreads) k_reduce(const float4* __restrict__ partial,
                                                const int64_t* __restrict__ pair_off,
                                                const int32_t* __restrict__ cnt, int64_t capacity, int n,
                                                ParamsIn P, float* __restrict__ g_means, float* __restrict__ g_chol,
                                                float* __restrict__ g_color, float* __restrict__ g_conic,
                                                AdamCfg cfg, float* __restrict__ params, float* __restrict__ m,
                                                float* __restrict__ v, float* __restrict__ grads_aos, Batch B,
                                                const double* __restrict__ loss_tile, double* __restrict__ loss) {
    __shared__ int s_step;
    // Adam: 1/(1 - b1^t), 1/sqrt(1 - b2^t); Adan: 1/(1 - b1^t), 1/(1 - b2^t),
    // 1/sqrt(1 - b3^t); [3] = learning-rate factor of the halving schedule.
    __shared__ float s_bc[4];
    pdl_wait();
    // The step counter's load is issued here and used after the partials are
    // summed, so no load below waits for it.
    int step_prev = 0;
    if (ADAM && threadIdx.x == 0) step_prev = *cfg.step;
    const int gblocks = (int)max(1, (n + kReduceThreads - 1) / kReduceThreads);
    // With loss_tile the first B.nimg blocks sum the images' squared errors
    // (first, so that they start in the first wave) and the Gaussian blocks
    // follow.
    const int lblocks = ADAM && loss_tile ? B.nimg : 0;
    const int gb = (int)blockIdx.x - lblocks;  // this block's index among the Gaussian blocks
    if (gb < 0) {
        // image b = blockIdx.x: its tiles' partials in tile order, eight loads
        // in flight per thread, combined in a fixed order, then a fixed
        // reduction tree (reproducible run to run); then the block counts
        // itself done like the others
        __shared__ double s_lw[32];
        {
            const int b = (int)blockIdx.x;
            const ImgDesc d = img_desc(B, b);
            const int nt = d.tw * d.th;
            double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            for (int i0 = threadIdx.x; i0 < nt; i0 += 8 * blockDim.x) {
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int i = i0 + u * blockDim.x;
                    if (i < nt) acc[u] += loss_tile[d.tile_base + i];
                }
            }
            double tot = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
            tot = block_sum<double>(tot, s_lw);
            if (threadIdx.x == 0) loss[b] = tot;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(cfg.done, 1u) == gridDim.x - 1) {
                *cfg.step = step_prev + 1;
                *cfg.done = 0u;
                __threadfence();
            }
        }
        return;
    }
    const int g = gb * blockDim.x + threadIdx.x;
    // Pair rows of the warp's 32 consecutive Gaussians are contiguous (emission
    // order): the warp streams them through shared memory with coalesced loads,
    // then each lane adds its own rows in emission order (Kahan), the same
    // order and arithmetic as reading them one by one.
    __shared__ float4 s_rows[kReduceThreads / 32][2][kReduceRows][2];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t p0 = 0, p1 = 0;
    int c = 0;
    if (g < n) {
        c = cnt[g];
        p0 = pair_off[g];
        p1 = min(p0 + (int64_t)c, capacity);
    }
    // Parameters and optimiser state do not depend on the partials: their
    // loads are issued first and overlap the staging below.
    float pp[8], mm[8], vv[8];
    float4* P4 = nullptr;
    float4* M4 = nullptr;
    float4* V4 = nullptr;
    if (ADAM && g < n) {
        P4 = reinterpret_cast<float4*>(params) + 2 * (size_t)g;
        M4 = reinterpret_cast<float4*>(m) + 2 * (size_t)g;
        V4 = reinterpret_cast<float4*>(v) + 2 * (size_t)g;
        *reinterpret_cast<float4*>(pp) = P4[0]; *reinterpret_cast<float4*>(pp + 4) = P4[1];
        *reinterpret_cast<float4*>(mm) = M4[0]; *reinterpret_cast<float4*>(mm + 4) = M4[1];
        *reinterpret_cast<float4*>(vv) = V4[0]; *reinterpret_cast<float4*>(vv + 4) = V4[1];
    }
    float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float ca[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    {
        const unsigned valid = __ballot_sync(0xffffffffu, g < n);
        if (valid) {
            const int64_t R0 = __shfl_sync(0xffffffffu, p0, __ffs(valid) - 1);
            const int64_t R1 = __shfl_sync(0xffffffffu, p1, 31 - __clz(valid));
            auto issue = [&](int64_t c0, int buf) {
                const int nr = (int)min((int64_t)kReduceRows, R1 - c0);
#pragma unroll
                for (int i = 0; i < kReduceRows / 32; ++i) {
                    const int r = lane + 32 * i;
                    if (r < nr) {
                        cp_async16(&s_rows[wid][buf][r][0], partial + 2 * (c0 + r));
                        cp_async16(&s_rows[wid][buf][r][1], partial + 2 * (c0 + r) + 1);
                    }
                }
                cp_async_commit();
            };
            issue(R0, 0);
            int buf = 0;
            for (int64_t c0 = R0; c0 < R1; c0 += kReduceRows, buf ^= 1) {
                const int nr = (int)min((int64_t)kReduceRows, R1 - c0);
                if (c0 + kReduceRows < R1) {
                    issue(c0 + kReduceRows, buf ^ 1);
                    cp_async_wait<1>();
                } else {
                    cp_async_wait<0>();
                }
                __syncwarp();
                const int64_t q1 = min(p1, c0 + nr);
                for (int64_t q = max(p0, c0); q < q1; ++q) {
                    const float4 u = s_rows[wid][buf][q - c0][0], w = s_rows[wid][buf][q - c0][1];
                    kahan_add(a[0], ca[0], u.x); kahan_add(a[1], ca[1], u.y);
                    kahan_add(a[2], ca[2], u.z); kahan_add(a[3], ca[3], u.w);
                    kahan_add(a[4], ca[4], w.x); kahan_add(a[5], ca[5], w.y);
                    kahan_add(a[6], ca[6], w.z); kahan_add(a[7], ca[7], w.w);
                }
                __syncwarp();
            }
        }
    }
    if (ADAM) {
        if (threadIdx.x == 0) {
            const int step = step_prev + 1;
            s_step = step;
            s_bc[0] = 1.f / (1.f - powf(cfg.beta1, (float)step));
            if (cfg.optimizer == 1) {
                s_bc[1] = 1.f / (1.f - powf(cfg.beta2, (float)step));
                s_bc[2] = rsqrtf(1.f - powf(cfg.beta3, (float)step));
            } else {
                s_bc[1] = rsqrtf(1.f - powf(cfg.beta2, (float)step));
                s_bc[2] = 0.f;
            }
            s_bc[3] = cfg.lr_halve_every > 0 ? ldexpf(1.f, -((step - 1) / cfg.lr_halve_every)) : 1.f;
        }
        __syncthreads();
    }
    // codec fine-tuning: this Gaussian's dL/dgamma, dL/dbeta terms, RVQ indices,
    // stage residuals and commitment term (zero when off or g >= n)
    float cv_gb[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int cv_j[kCodecMaxStages] = {-1, -1, -1, -1};
    float cv_r[kCodecMaxStages][3] = {};
    float cv_commit = 0.f;
    if (g < n) {
        float l1 = P.chol[(int64_t)g * P.ls], l2 = P.chol[(int64_t)g * P.ls + 1], l3 = P.chol[(int64_t)g * P.ls + 2];
        const bool rs_mode = ADAM && cfg.cov_mode == 1;
        if (ADAM && cfg.param_mode == 1) {  // App. C.1: +0.5 on the Cholesky diagonal or on the scales
            if (rs_mode) {
                l2 += 0.5f;
                l3 += 0.5f;
            } else {
                l1 += 0.5f;
                l3 += 0.5f;
            }
        }
        constexpr bool codec = ADAM && CODEC;
        float cx[3] = {0.f, 0.f, 0.f}, cq[3] = {0.f, 0.f, 0.f};
        if constexpr (codec) {  // the render saw the quantised Cholesky vector (Sec. 3.3)
            const CodecCfg& Q = B.codec;
            l1 = lsq_quant(l1, Q.gb[0], Q.gb[3], Q.qp, cx[0], cq[0]);
            l2 = lsq_quant(l2, Q.gb[1], Q.gb[4], Q.qp, cx[1], cq[1]);
            l3 = lsq_quant(l3, Q.gb[2], Q.gb[5], Q.qp, cx[2], cq[2]);
        }
#pragma unroll
        for (int s = 0; s < 8; ++s) a[s] -= ca[s];
        float gr[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        float gq[3] = {0.f, 0.f, 0.f};
        if (c > 0) {
            // Sigma: from the Cholesky vector, or in the rotation-scaling form
            // (slots theta, s1, s2) from (R S)(R S)^T with det = (s1 s2)^2.
            float s11, s12, s22, det, rc = 0.f, rsn = 0.f;
            if (rs_mode) {
                sincosf(l1, &rsn, &rc);
                const float q1 = l2 * l2, q2 = l3 * l3, ds = l2 * l3;
                s11 = rc * rc * q1 + rsn * rsn * q2;
                s12 = rc * rsn * (q1 - q2);
                s22 = rsn * rsn * q1 + rc * rc * q2;
                det = ds * ds;
            } else {
                s11 = l1 * l1;
                s12 = l1 * l2;
                s22 = l2 * l2 + l3 * l3;
                const float dd = l1 * l3;
                det = dd * dd;
            }
            const float A = s22 / det, Bc = -s12 / det, C = s11 / det;
            const float Sx = a[3], Sy = a[4], Sxx = a[5], Sxy = a[6], Syy = a[7];
            const float gA = -0.5f * Sxx, gB = -Sxy, gC = -0.5f * Syy;
            gq[0] = gA; gq[1] = gB; gq[2] = gC;
            gr[0] = A * Sx + Bc * Sy;
            gr[1] = Bc * Sx + C * Sy;
            const float h = 0.5f * gB;
            const float QG11 = A * gA + Bc * h, QG12 = A * h + Bc * gC;
            const float QG21 = Bc * gA + C * h, QG22 = Bc * h + C * gC;
            const float g1 = -(QG11 * A + QG12 * Bc);
            const float g2 = -(QG11 * Bc + QG12 * C);
            const float g3 = -(QG21 * Bc + QG22 * C);
            if (rs_mode) {
                // dL/dx = g1 dSigma11/dx + 2 g2 dSigma12/dx + g3 dSigma22/dx, x = theta, s1, s2
                const float q1 = l2 * l2, q2 = l3 * l3, cs2 = 2.f * rc * rsn;
                gr[2] = cs2 * (q2 - q1) * g1 + 2.f * g2 * (rc * rc - rsn * rsn) * (q1 - q2) + cs2 * (q1 - q2) * g3;
                gr[3] = 2.f * l2 * (rc * rc * g1 + 2.f * rc * rsn * g2 + rsn * rsn * g3);
                gr[4] = 2.f * l3 * (rsn * rsn * g1 - 2.f * rc * rsn * g2 + rc * rc * g3);
            } else {
                gr[2] = 2.f * (g1 * l1 + g2 * l2);
                gr[3] = 2.f * (g2 * l1 + g3 * l2);
                gr[4] = 2.f * g3 * l3;
            }
            gr[5] = a[0]; gr[6] = a[1]; gr[7] = a[2];
        }
        if (!ADAM) {
            if (g_means) { g_means[2 * g] = gr[0]; g_means[2 * g + 1] = gr[1]; }
            if (g_chol) { g_chol[3 * g] = gr[2]; g_chol[3 * g + 1] = gr[3]; g_chol[3 * g + 2] = gr[4]; }
            if (g_color) { g_color[3 * g] = gr[5]; g_color[3 * g + 1] = gr[6]; g_color[3 * g + 2] = gr[7]; }
            if (g_conic) { g_conic[3 * g] = gq[0]; g_conic[3 * g + 1] = gq[1]; g_conic[3 * g + 2] = gq[2]; }
        } else {
            if constexpr (codec) {
                // Straight-through gradients (Sec. 3.3): FP16 positions and RVQ
                // colour pass dL/d(quantised) unchanged; the quantiser passes it
                // inside its range and feeds gamma, beta (the LSQ+ convention).
                const float qp = B.codec.qp;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const float gi = gr[2 + i];
                    const bool inside = cx[i] >= 0.f && cx[i] <= qp, outside = cx[i] < 0.f || cx[i] > qp;
                    cv_gb[i] = inside ? gi * (cq[i] - cx[i]) : (cx[i] > qp ? gi * qp : 0.f);
                    cv_gb[3 + i] = outside ? gi : 0.f;
                    gr[2 + i] = inside ? gi : 0.f;
                }
                // RVQ residuals each stage quantised, for the EMA codebook update
                // and the commitment loss (Eq. 11).
                const CodecCfg& Q = B.codec;
                float r0 = pp[5], r1 = pp[6], r2 = pp[7];
#pragma unroll
                for (int mm_ = 0; mm_ < kCodecMaxStages; ++mm_) {
                    if (mm_ < Q.stages) {
                        const int j = Q.idx[(size_t)mm_ * B.total_gauss + g];
                        const float* e = Q.codebooks + ((size_t)mm_ * Q.size + j) * 3;
                        cv_j[mm_] = j;
                        cv_r[mm_][0] = r0; cv_r[mm_][1] = r1; cv_r[mm_][2] = r2;
                        r0 = __fsub_rn(r0, e[0]);
                        r1 = __fsub_rn(r1, e[1]);
                        r2 = __fsub_rn(r2, e[2]);
                        cv_commit += r0 * r0 + r1 * r1 + r2 * r2;
                    }
                }
            }
            float g_logit = 0.f;
            if constexpr (OPAC > 0) {
                // Separate opacity o = sigmoid(logit): accumulated summation
                // rendered c' = c o, so dL/dc = dL/dc' o and dL/do = dL/dc' . c;
                // alpha-blending summed dL/do per pair (ninth sum).
                const float o = B.opac.o[g];
                float dldo;
                if constexpr (OPAC == 1) {
                    dldo = gr[5] * pp[5] + gr[6] * pp[6] + gr[7] * pp[7];
                    gr[5] *= o;
                    gr[6] *= o;
                    gr[7] *= o;
                } else {
                    float s = 0.f, cs = 0.f;
                    for (int64_t q = p0; q < p1; ++q) kahan_add(s, cs, B.opac.partial[q]);
                    dldo = s - cs;
                }
                g_logit = c > 0 ? dldo * o * (1.f - o) : 0.f;
                B.opac.grad[g] = g_logit;
                float lm = B.opac.m[g], lv = B.opac.v[g];
                B.opac.logit[g] = opt_step(cfg, s_bc, s_step, cfg.lr[2] * s_bc[3], g_logit, B.opac.logit[g], lm, lv,
                                           B.opac.n + g, B.opac.gp + g);
                B.opac.m[g] = lm;
                B.opac.v[g] = lv;
            }
            if (cfg.param_mode == 1 && c > 0) {
                // d mu / d theta = (1 - tanh^2(theta)) / 2 * (W, H)
                const ImgDesc d = img_desc(B, image_of_gauss(B, g));
                const float tx = tanhf(pp[0]), ty = tanhf(pp[1]);
                gr[0] *= (1.f - tx) * (1.f + tx) * 0.5f * (float)d.W;
                gr[1] *= (1.f - ty) * (1.f + ty) * 0.5f * (float)d.H;
            }
            if (grads_aos) {
                float4* go = reinterpret_cast<float4*>(grads_aos) + 2 * (size_t)g;
                go[0] = make_float4(gr[0], gr[1], gr[2], gr[3]);
                go[1] = make_float4(gr[4], gr[5], gr[6], gr[7]);
            }
            if (cfg.optimizer == 1) {
                // Adan (Xie et al. 2022), no weight decay: m, v, n average the
                // gradient, its change and the square of the extrapolated
                // gradient g + b2 (g - g_prev); the first step takes g_prev = g.
                float nn[8], gp[8];
                float4* N4 = reinterpret_cast<float4*>(cfg.n) + 2 * (size_t)g;
                float4* G4 = reinterpret_cast<float4*>(cfg.g_prev) + 2 * (size_t)g;
                *reinterpret_cast<float4*>(nn) = N4[0]; *reinterpret_cast<float4*>(nn + 4) = N4[1];
                *reinterpret_cast<float4*>(gp) = G4[0]; *reinterpret_cast<float4*>(gp + 4) = G4[1];
#pragma unroll
                for (int s = 0; s < 8; ++s) {
                    const float lr = cfg.lr[s < 2 ? 0 : (s < 5 ? 1 : 2)] * s_bc[3];
                    const float dg = s_step == 1 ? 0.f : gr[s] - gp[s];
                    mm[s] = cfg.beta1 * mm[s] + (1.f - cfg.beta1) * gr[s];
                    vv[s] = cfg.beta2 * vv[s] + (1.f - cfg.beta2) * dg;
                    const float ge = gr[s] + cfg.beta2 * dg;
                    nn[s] = cfg.beta3 * nn[s] + (1.f - cfg.beta3) * ge * ge;
                    const float dir = mm[s] * s_bc[0] + cfg.beta2 * (vv[s] * s_bc[1]);
                    pp[s] -= lr * dir / (sqrtf(nn[s]) * s_bc[2] + cfg.eps);
                    gp[s] = gr[s];
                }
                N4[0] = *reinterpret_cast<float4*>(nn); N4[1] = *reinterpret_cast<float4*>(nn + 4);
                G4[0] = *reinterpret_cast<float4*>(gp); G4[1] = *reinterpret_cast<float4*>(gp + 4);
            } else {
#pragma unroll
                for (int s = 0; s < 8; ++s) {
                    const float lr = cfg.lr[s < 2 ? 0 : (s < 5 ? 1 : 2)] * s_bc[3];
                    mm[s] = cfg.beta1 * mm[s] + (1.f - cfg.beta1) * gr[s];
                    vv[s] = cfg.beta2 * vv[s] + (1.f - cfg.beta2) * gr[s] * gr[s];
                    const float denom = sqrtf(vv[s]) * s_bc[1] + cfg.eps;
                    pp[s] -= (lr * s_bc[0]) * mm[s] / denom;
                }
            }
            P4[0] = *reinterpret_cast<float4*>(pp); P4[1] = *reinterpret_cast<float4*>(pp + 4);
            M4[0] = *reinterpret_cast<float4*>(mm); M4[1] = *reinterpret_cast<float4*>(mm + 4);
            V4[0] = *reinterpret_cast<float4*>(vv); V4[1] = *reinterpret_cast<float4*>(vv + 4);
        }
    }
    if (ADAM && CODEC) codec_block_partials(B.codec, cv_gb, cv_j, cv_r, cv_commit, gb, gblocks);
    if (ADAM) {
        // The last block to finish advances the step counter (every block has
        // read it by then).
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned prev = atomicAdd(cfg.done, 1u);
            if (prev == gridDim.x - 1) {
                *cfg.step = s_step;
                *cfg.done = 0u;
                __threadfence();
            }
        }
    }
}

// Codec sums, stage 2: block v adds row v of the per-block partials in a
// fixed order (thread t takes blocks t, t + 256, ...; then a fixed tree), so
// the result is reproducible. The last block to finish applies the sums:
// the optimiser step of gamma, beta (the same optimiser and bias
// corrections as the Gaussians, the Cholesky learning rate), the EMA
// codebook update (Sec. 3.4) and the commitment loss L_c (Eq. 11).
constexpr int kCodecSumThreads = 256;

__global__ void __launch_bounds__(kCodecSumThreads) k_codec_update(CodecCfg Q, AdamCfg cfg, int nblocks, int n) {
    double* tot = Q.tot;
    unsigned* ticket = Q.ticket;
    __shared__ double s_w[32];
    __shared__ bool s_last;
    pdl_wait();
    const int v = blockIdx.x;
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) acc += Q.part[(size_t)v * nblocks + b];
    acc = block_sum<double>(acc, s_w);
    if (threadIdx.x == 0) {
        tot[v] = acc;
        __threadfence();
        s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int nv = codec_nvals(Q);
    const int t = threadIdx.x;
    // Everything the update reads is loaded in parallel first (a chain of
    // dependent global read-modify-writes would cost a round trip each).
    constexpr int kMB = kCodecMaxEntries;
    __shared__ double s_tot[kCodecMaxVals];
    __shared__ double s_cnt[kMB];
    __shared__ double s_sum[kMB * 3];
    __shared__ double s_stage[kCodecMaxStages];
    const int MB = Q.stages * Q.size;
    for (int i = t; i < nv; i += blockDim.x) s_tot[i] = __ldcg(tot + i);
    for (int i = t; i < MB; i += blockDim.x) s_cnt[i] = Q.ema_count[i];
    for (int i = t; i < 3 * MB; i += blockDim.x) s_sum[i] = Q.ema_total[i];
    __syncthreads();
    {
        const double d = (double)Q.decay;
        for (int i = t; i < MB; i += blockDim.x) {
            const double c = d * s_cnt[i] + (1.0 - d) * s_tot[6 + 4 * i];
            s_cnt[i] = c;
            Q.ema_count[i] = c;
            for (int k = 0; k < 3; ++k) {
                const double s = d * s_sum[3 * i + k] + (1.0 - d) * s_tot[6 + 4 * i + 1 + k];
                s_sum[3 * i + k] = s;
                Q.ema_total[3 * i + k] = s;
            }
        }
    }
    __syncthreads();
    if (t < Q.stages) {
        double sum = 0.0;
        for (int j = 0; j < Q.size; ++j) sum += s_cnt[t * Q.size + j];
        s_stage[t] = sum;
    }
    __syncthreads();
    for (int i = t; i < 3 * MB; i += blockDim.x) {
        const int e = i / 3, st = e / Q.size;
        const double e_ = (double)Q.eps, sum = s_stage[st];
        const double sm = (s_cnt[e] + e_) / (sum + Q.size * e_) * sum;
        Q.codebooks[i] = (float)(s_sum[i] / sm);
    }
    if (t < 6) {
        const float gr = (float)s_tot[t];
        Q.out[1 + t] = s_tot[t];
        const int step = *cfg.step;  // already advanced by the reduction
        const float lr = cfg.lr[1] * (cfg.lr_halve_every > 0 ? ldexpf(1.f, -((step - 1) / cfg.lr_halve_every)) : 1.f);
        float* p = Q.gb;
        float& m = p[6 + t];
        float& vv = p[12 + t];
        if (cfg.optimizer == 1) {
            float& nn = p[18 + t];
            float& gp = p[24 + t];
            const float dg = step == 1 ? 0.f : gr - gp;
            m = cfg.beta1 * m + (1.f - cfg.beta1) * gr;
            vv = cfg.beta2 * vv + (1.f - cfg.beta2) * dg;
            const float ge = gr + cfg.beta2 * dg;
            nn = cfg.beta3 * nn + (1.f - cfg.beta3) * ge * ge;
            const float b1 = 1.f / (1.f - powf(cfg.beta1, (float)step)), b2 = 1.f / (1.f - powf(cfg.beta2, (float)step));
            const float b3 = rsqrtf(1.f - powf(cfg.beta3, (float)step));
            p[t] -= lr * (m * b1 + cfg.beta2 * (vv * b2)) / (sqrtf(nn) * b3 + cfg.eps);
            gp = gr;
        } else {
            m = cfg.beta1 * m + (1.f - cfg.beta1) * gr;
            vv = cfg.beta2 * vv + (1.f - cfg.beta2) * gr * gr;
            const float b1 = 1.f / (1.f - powf(cfg.beta1, (float)step)), b2 = rsqrtf(1.f - powf(cfg.beta2, (float)step));
            p[t] -= (lr * b1) * m / (sqrtf(vv) * b2 + cfg.eps);
        }
    } else if (t == 64) {
        Q.out[0] = n > 0 ? s_tot[nv - 1] / ((double)n * Q.size) : 0.0;
        *ticket = 0u;
    }
}

}  // namespace

namespace {

// Resident blocks per SM of a kernel at its launch shape (cached per device).
template <int T>
int backward_blocks_per_sm() {
    static std::mutex mu;
    static std::map<int, int> cached;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    std::lock_guard<std::mutex> lk(mu);
    int& v = cached[dev];
    if (v <= 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_backward<T>, kBwdThreads, backward_smem<T>()) !=
                cudaSuccess ||
            nb <= 0)
            nb = 1;
        v = nb;
    }
    return v;
}

template <int T>
cudaError_t launch_backward_t(const float4* rec_binned, const uint32_t* keys, const uint32_t* emit,
                              const float* dl_tiled, const Batch& B, const int64_t* k_dev, int64_t capacity,
                              float4* partial, uint32_t* status, cudaStream_t s) {
    cudaError_t e = smem_optin(reinterpret_cast<const void*>(k_backward<T>), (int)backward_smem<T>());
    if (e != cudaSuccess) return e;
    // persistent: one wave of resident blocks (no more than the tasks need)
    const int64_t tasks = (capacity + 31) / 32;
    const int64_t full = (int64_t)sm_count() * backward_blocks_per_sm<T>();
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(full, (tasks + kBwdWarps - 1) / kBwdWarps));
    return launch_pdl(k_backward<T>, dim3(blocks), dim3(kBwdThreads), backward_smem<T>(), s, rec_binned, keys, emit,
                      dl_tiled, B, k_dev, capacity, partial, status);
}

}  // namespace

cudaError_t launch_backward(const float4* rec_binned, const uint32_t* keys, const uint32_t* emit,
                            const float* dl_tiled, const Batch& B, const int64_t* k_dev, int64_t capacity,
                            float4* partial, uint32_t* status, cudaStream_t s) {
    if (capacity <= 0) return cudaSuccess;
    switch (B.tile) {
        case 8: return launch_backward_t<8>(rec_binned, keys, emit, dl_tiled, B, k_dev, capacity, partial, status, s);
        case 16: return launch_backward_t<16>(rec_binned, keys, emit, dl_tiled, B, k_dev, capacity, partial, status, s);
        case 32: return launch_backward_t<32>(rec_binned, keys, emit, dl_tiled, B, k_dev, capacity, partial, status, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_emit_index(const uint32_t* keys, const uint32_t* ids, const int4* rect, const int64_t* pair_off,
                              const Batch& B, const int64_t* k_dev, int64_t capacity, uint32_t* emit, uint32_t* status,
                              cudaStream_t s) {
    if (capacity <= 0) return cudaSuccess;
    const int blocks = std::max(1, std::min<int>(sm_count() * 8, (int)((capacity + 255) / 256)));
    return launch_pdl(k_emit_index, dim3(blocks), dim3(256), 0, s, keys, ids, rect, pair_off, B, k_dev, capacity, emit,
                      status);
}

cudaError_t launch_pack_dl(const float* dl_hwc, const Batch& B, float* dl_tiled, cudaStream_t s) {
    if (B.total_tiles <= 0) return cudaSuccess;
    switch (B.tile) {
        case 8: return launch_pdl(k_pack_dl<8>, dim3(B.total_tiles), dim3(64), 0, s, dl_hwc, B, dl_tiled);
        case 16: return launch_pdl(k_pack_dl<16>, dim3(B.total_tiles), dim3(256), 0, s, dl_hwc, B, dl_tiled);
        case 32: return launch_pdl(k_pack_dl<32>, dim3(B.total_tiles), dim3(256), 0, s, dl_hwc, B, dl_tiled);
        default: return cudaErrorInvalidValue;
    }
}

int64_t reduce_blocks(int64_t n) { return std::max<int64_t>(1, (n + kReduceThreads - 1) / kReduceThreads); }

cudaError_t launch_reduce(const float4* partial, const int64_t* pair_off, const int32_t* cnt, int64_t capacity,
                          int32_t n, const ParamsIn& P, float* g_means, float* g_chol, float* g_color,
                          float* g_conic, const AdamCfg* adam, float* params, float* m, float* v, float* grads_aos,
                          const Batch& B, cudaStream_t s, const double* loss_tile, double* loss) {
    const int blocks = (int)reduce_blocks(n);
    if (adam) {
        const bool codec = B.codec.bits > 0;
        auto kern = codec ? k_reduce<true, true, 0>
                          : (B.opac.mode == 1 ? k_reduce<true, false, 1>
                                              : (B.opac.mode == 2 ? k_reduce<true, false, 2> : k_reduce<true, false, 0>));
        // codec: the per-warp sums of every codebook entry in dynamic shared memory
        const int nv = 6 + B.codec.stages * B.codec.size * 4 + 1;
        const size_t dyn = codec ? (size_t)(kReduceThreads / 32) * nv * sizeof(float) : 0;
        if (codec) {
            cudaError_t e0 = smem_optin(reinterpret_cast<const void*>(kern), (int)dyn);
            if (e0 != cudaSuccess) return e0;
        }
        // one more block per image sums its squared error when loss_tile is given
        const int grid = blocks + (loss_tile ? B.nimg : 0);
        cudaError_t e = launch_pdl(kern, dim3(grid), dim3(kReduceThreads), dyn, s, partial, pair_off, cnt, capacity, n,
                                   P, (float*)nullptr, (float*)nullptr, (float*)nullptr, (float*)nullptr, *adam, params,
                                   m, v, grads_aos, B, loss_tile, loss);
        if (e != cudaSuccess || B.codec.bits == 0) return e;
        return launch_pdl(k_codec_update, dim3(nv), dim3(kCodecSumThreads), 0, s, B.codec, *adam, blocks, n);
    }
    AdamCfg none{};
    return launch_pdl(k_reduce<false>, dim3(blocks), dim3(kReduceThreads), 0, s, partial, pair_off, cnt, capacity, n, P,
                      g_means, g_chol, g_color, g_conic, none, (float*)nullptr, (float*)nullptr, (float*)nullptr,
                      (float*)nullptr, B, (const double*)nullptr, (double*)nullptr);
}

}  // namespace gi
