// blend.cu -- sorted alpha-blending render and its gradients (Sec. 3.2,
// Eq. 3-4): the rasterisation that accumulated summation replaces, built to
// measure that replacement on the same hardware (Table 3's "w/o AR").
//
//   alpha_n = min(0.99, o_n exp(-sigma_n)), skipped when alpha_n < 1/255,
//   C_i = sum_n c_n alpha_n T_n, T_n = prod_{m < n} (1 - alpha_m),
//   the walk stopping before the Gaussian that would take T below 1e-4
//
// over each tile's list in ascending Gaussian index (a 2D image has no depth
// to sort by). One CTA per 16 x 16 tile, a few pixels per thread: the list is
// staged through shared memory in chunks and every pixel walks it front to
// back, the CTA stopping once all its pixels have saturated.
//
// Gradients, per pixel and front to back again with the same operations
// (so the same decisions), using the final colour C from the forward pass:
// with the prefix P_n = sum_{m <= n} c_m alpha_m T_m and the suffix
// S = C - P_n,
//   dL/dc_n     = sum_i dL/dC_i alpha_n T_n
//   dL/dalpha_n = sum_ch dL/dC (c_n T_n - S / (1 - alpha_n))
// and, unless alpha_n was clamped, dL/dsigma_n = -dL/dalpha_n alpha_n and
// dL/do_n = dL/dalpha_n exp(-sigma_n). The per-pixel terms of each list entry
// are summed over the tile's 256 pixels (a thread's pixels in registers, warp
// butterflies, then the warps in order) into the same eight per-pair sums the accumulated backward writes
// (colour, and e~ (dx, dy, dx^2, dx dy, dy^2) with e~ = -dL/dsigma) plus a
// ninth for the opacity, at the pair's emission index; the per-Gaussian
// reduction is then shared with the accumulated path. Deterministic.
#include "kernels.cuh"

namespace gi {
namespace {

constexpr int kBT = 16;
constexpr int kBPix = kBT * kBT;
constexpr int kBWarps = kBPix / 32;
constexpr int kBChunk = 32;  // list entries per backward chunk
#ifndef GI_BLEND_RENDER_PX
#define GI_BLEND_RENDER_PX 2
#endif
#ifndef GI_BLEND_BACKWARD_PX
#define GI_BLEND_BACKWARD_PX 4
#endif
constexpr int kBlendRenderPx = GI_BLEND_RENDER_PX;      // pixels per thread, forward
constexpr int kBlendBackwardPx = GI_BLEND_BACKWARD_PX;  // pixels per thread, backward

// exp(-sigma) of a record at a pixel centre, with explicit roundings so the
// forward and the backward kernel compute the same value.
__device__ __forceinline__ float blend_w(const float4 r0, const float4 r1, float px, float py, float& dx,
                                         float& dy) {
    dx = __fsub_rn(px, r0.x);
    dy = __fsub_rn(py, r0.y);
    const float z1 = __fmul_rn(r0.z, dx);
    const float z2 = __fadd_rn(__fmul_rn(r0.w, dx), __fmul_rn(r1.x, dy));
    return ex2(-__fadd_rn(__fmul_rn(z1, z1), __fmul_rn(z2, z2)));
}

// Reduce-scatter of 16 per-lane values over the warp (16 shuffles instead of
// 16 x 5): after the call, lanes 2s and 2s + 1 both hold the warp sum of slot
// s in v[0]. Fixed order, so deterministic.
__device__ __forceinline__ void warp_reduce_scatter16(float (&v)[16], int lane) {
#pragma unroll
    for (int w = 8; w >= 1; w >>= 1) {  // offsets 16, 8, 4, 2: keep w slots
        const int off = 2 * w;
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < w; ++i) {
            const float send = up ? v[i] : v[i + w];
            const float keep = up ? v[i + w] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
}

struct TileGeo {
    ImgDesc d;
    int img, tx, ty, b, e;
};

__device__ __forceinline__ TileGeo tile_geo(const Batch& B, const int2* ranges, int t, uint32_t* status) {
    TileGeo g;
    g.img = image_of_tile(B, t);
    g.d = img_desc(B, g.img);
    const int lt = t - g.d.tile_base;
    g.tx = lt % g.d.tw;
    g.ty = lt / g.d.tw;
    const int2 rg = ranges[t];
    const bool ok = gi_in_bounds(rg.x >= 0 && rg.x <= rg.y, status);
    g.b = ok ? rg.x : 0;
    g.e = ok ? rg.y : 0;
    return g;
}

// PX pixels per thread (rows tid / 16 + i * NT / 16): each staged record is
// read from shared memory once per thread and applied to all its pixels.
template <int PX>
__global__ void __launch_bounds__(kBPix / PX) k_render_blend(const float4* __restrict__ rec_binned,
                                                             const uint32_t* __restrict__ ids,
                                                             const float* __restrict__ o_eff,
                                                             const int2* __restrict__ ranges, Batch B,
                                                             const float* __restrict__ target,
                                                             float* __restrict__ out, int32_t* __restrict__ n_last,
                                                             float* __restrict__ dl_tiled,
                                                             double* __restrict__ loss_sum, uint32_t* status) {
    constexpr int NT = kBPix / PX;
    constexpr int kStage = 256;  // list entries staged per chunk
    __shared__ float4 s_rec[kStage][2];
    __shared__ float s_o[kStage];
    __shared__ float s_red[32];
    pdl_wait();
    const int t = blockIdx.x;
    const TileGeo tg = tile_geo(B, ranges, t, status);
    const ImgDesc& d = tg.d;
    const int tid = threadIdx.x;
    float px[PX], py[PX], C0[PX], C1[PX], C2[PX], Tr[PX];
    int last[PX];
    unsigned done = 0u;  // bit i: pixel i has stopped (or lies outside the image)
#pragma unroll
    for (int i = 0; i < PX; ++i) {
        const int q = tid + NT * i;
        const int x = tg.tx * kBT + q % kBT, y = tg.ty * kBT + q / kBT;
        px[i] = (float)x + 0.5f;
        py[i] = (float)y + 0.5f;
        C0[i] = C1[i] = C2[i] = 0.f;
        Tr[i] = 1.f;
        last[i] = 0;
        if (!(x < d.W && y < d.H)) done |= 1u << i;
    }
    constexpr unsigned kAll = (1u << PX) - 1u;
    for (int base = tg.b; base < tg.e; base += kStage) {
        if (__syncthreads_and(done == kAll)) break;  // also orders the restaging after the last chunk's reads
        for (int s = tid; s < kStage; s += NT) {
            const int k = base + s;
            if (k < tg.e) {
                uint32_t g = ids[k];
                if (!gi_in_bounds(g < (uint32_t)B.total_gauss, status)) g = 0;
                s_rec[s][0] = rec_binned[2 * (size_t)k];
                s_rec[s][1] = rec_binned[2 * (size_t)k + 1];
                s_o[s] = o_eff[g];
            }
        }
        __syncthreads();
        const int n = min(kStage, tg.e - base);
        for (int j = 0; j < n && done != kAll; ++j) {
            const float4 r0 = s_rec[j][0], r1 = s_rec[j][1];
            const float o = s_o[j];
#pragma unroll
            for (int i = 0; i < PX; ++i) {
                if (done & (1u << i)) continue;
                float dx, dy;
                const float w = blend_w(r0, r1, px[i], py[i], dx, dy);
                float a = __fmul_rn(o, w);
                if (a < kBlendAlphaMin) continue;
                a = fminf(a, kBlendAlphaMax);
                const float test = __fmul_rn(Tr[i], __fsub_rn(1.f, a));
                if (test < kBlendTMin) {
                    done |= 1u << i;
                    continue;
                }
                const float at = __fmul_rn(a, Tr[i]);
                C0[i] = __fadd_rn(C0[i], __fmul_rn(r1.y, at));
                C1[i] = __fadd_rn(C1[i], __fmul_rn(r1.z, at));
                C2[i] = __fadd_rn(C2[i], __fmul_rn(r1.w, at));
                Tr[i] = test;
                last[i] = base - tg.b + j + 1;
            }
        }
    }
    const float scale = 2.0f / (3.0f * (float)d.W * (float)d.H);
    float lsum = 0.f;
#pragma unroll
    for (int i = 0; i < PX; ++i) {
        const int q = tid + NT * i;
        const int x = tg.tx * kBT + q % kBT, y = tg.ty * kBT + q / kBT;
        float dl0 = 0.f, dl1 = 0.f, dl2 = 0.f;
        if (x < d.W && y < d.H) {
            const int64_t pix = d.pix_base + (int64_t)y * d.W + x;
            out[3 * pix] = C0[i];
            out[3 * pix + 1] = C1[i];
            out[3 * pix + 2] = C2[i];
            if (n_last) n_last[pix] = last[i];
            if (target) {
                const float r0 = C0[i] - target[3 * pix], r1 = C1[i] - target[3 * pix + 1],
                            r2 = C2[i] - target[3 * pix + 2];
                lsum = fmaf(r2, r2, fmaf(r1, r1, fmaf(r0, r0, lsum)));
                dl0 = r0 * scale;
                dl1 = r1 * scale;
                dl2 = r2 * scale;
            }
        }
        if (dl_tiled) {  // planar per tile, as the accumulated render writes it
            float* dt = dl_tiled + (size_t)t * 3 * kBPix;
            dt[q] = dl0;
            dt[kBPix + q] = dl1;
            dt[2 * kBPix + q] = dl2;
        }
    }
    if (target && loss_sum) {
        lsum = warp_sum(lsum);
        if ((tid & 31) == 0) s_red[tid >> 5] = lsum;
        __syncthreads();
        if (tid == 0) {
            float s = 0.f;
            for (int w = 0; w < NT / 32; ++w) s += s_red[w];
            atomicAdd(&loss_sum[tg.img], (double)s);
        }
    }
}

// Emission index of pair (tile tx, ty; Gaussian g): pair_off[g] plus the
// tile's row-major rank inside g's rect; -1 when out of range.
__device__ __forceinline__ int64_t emission_index(const int4* rect, const int64_t* pair_off, uint32_t g, int tx,
                                                  int ty, int64_t capacity) {
    const int4 r = rect[g];
    const int64_t e = pair_off[g] + (int64_t)(ty - r.y) * (r.z - r.x) + (tx - r.x);
    return (e >= 0 && e < capacity) ? e : -1;
}

template <int PX>
__global__ void __launch_bounds__(kBPix / PX) k_backward_blend(
    const float4* __restrict__ rec_binned, const uint32_t* __restrict__ ids, const float* __restrict__ o_eff,
    const int2* __restrict__ ranges, const int4* __restrict__ rect, const int64_t* __restrict__ pair_off, Batch B,
    const float* __restrict__ out, const int32_t* __restrict__ n_last, const float* __restrict__ dl_tiled,
    int64_t capacity, float* __restrict__ partial, float* __restrict__ partial_o, uint32_t* status) {
    constexpr int NT = kBPix / PX, NW = NT / 32;
    __shared__ float4 s_rec[kBChunk][2];
    __shared__ float s_o[kBChunk];
    __shared__ int64_t s_e[kBChunk];
    __shared__ float s_red[kBChunk][NW][9];
    __shared__ int s_max[NW];
    pdl_wait();
    const int t = blockIdx.x;
    const TileGeo tg = tile_geo(B, ranges, t, status);
    const ImgDesc& d = tg.d;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float* dt = dl_tiled + (size_t)t * 3 * kBPix;
    float px[PX], py[PX], g0[PX], g1[PX], g2[PX], Cf0[PX], Cf1[PX], Cf2[PX], P0[PX], P1[PX], P2[PX], Tr[PX];
    int nl[PX];
    int mine = 0;
#pragma unroll
    for (int i = 0; i < PX; ++i) {
        const int q = tid + NT * i;
        const int x = tg.tx * kBT + q % kBT, y = tg.ty * kBT + q / kBT;
        px[i] = (float)x + 0.5f;
        py[i] = (float)y + 0.5f;
        g0[i] = dt[q];
        g1[i] = dt[kBPix + q];
        g2[i] = dt[2 * kBPix + q];
        Cf0[i] = Cf1[i] = Cf2[i] = 0.f;
        nl[i] = 0;
        if (x < d.W && y < d.H) {
            const int64_t pix = d.pix_base + (int64_t)y * d.W + x;
            Cf0[i] = out[3 * pix];
            Cf1[i] = out[3 * pix + 1];
            Cf2[i] = out[3 * pix + 2];
            nl[i] = min(n_last[pix], tg.e - tg.b);
        }
        P0[i] = P1[i] = P2[i] = 0.f;
        Tr[i] = 1.f;
        mine = max(mine, nl[i]);
    }
    {
        const int m = __reduce_max_sync(0xffffffffu, mine);
        if (lane == 0) s_max[warp] = m;
    }
    __syncthreads();
    int nmax = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) nmax = max(nmax, s_max[w]);
    for (int base = tg.b; base < tg.b + nmax; base += kBChunk) {
        const int n = min(kBChunk, tg.b + nmax - base);
        if (tid < n) {
            const int k = base + tid;
            uint32_t g = ids[k];
            const bool ok = gi_in_bounds(g < (uint32_t)B.total_gauss, status);
            if (!ok) g = 0;
            s_rec[tid][0] = rec_binned[2 * (size_t)k];
            s_rec[tid][1] = rec_binned[2 * (size_t)k + 1];
            s_o[tid] = o_eff[g];
            s_e[tid] = ok ? emission_index(rect, pair_off, g, tg.tx, tg.ty, capacity) : -1;
        }
        __syncthreads();
        for (int j = 0; j < n; ++j) {
            const float4 r0 = s_rec[j][0], r1 = s_rec[j][1];
            const float o = s_o[j];
            const int pos = base - tg.b + j;
            float v[16] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int i = 0; i < PX; ++i) {
                if (pos >= nl[i]) continue;
                float dx, dy;
                const float w = blend_w(r0, r1, px[i], py[i], dx, dy);
                float a = __fmul_rn(o, w);
                if (a < kBlendAlphaMin) continue;
                const bool clamped = a > kBlendAlphaMax;
                a = fminf(a, kBlendAlphaMax);
                const float at = __fmul_rn(a, Tr[i]);
                P0[i] = __fadd_rn(P0[i], __fmul_rn(r1.y, at));
                P1[i] = __fadd_rn(P1[i], __fmul_rn(r1.z, at));
                P2[i] = __fadd_rn(P2[i], __fmul_rn(r1.w, at));
                const float inv = __fdividef(1.f, 1.f - a);
                const float dla = g0[i] * (r1.y * Tr[i] - (Cf0[i] - P0[i]) * inv) +
                                  g1[i] * (r1.z * Tr[i] - (Cf1[i] - P1[i]) * inv) +
                                  g2[i] * (r1.w * Tr[i] - (Cf2[i] - P2[i]) * inv);
                v[0] = fmaf(g0[i], at, v[0]);
                v[1] = fmaf(g1[i], at, v[1]);
                v[2] = fmaf(g2[i], at, v[2]);
                if (!clamped) {
                    const float ee = dla * a;  // -dL/dsigma
                    const float ex = ee * dx, ey = ee * dy;
                    v[3] += ex;
                    v[4] += ey;
                    v[5] = fmaf(ex, dx, v[5]);
                    v[6] = fmaf(ex, dy, v[6]);
                    v[7] = fmaf(ey, dy, v[7]);
                    v[8] = fmaf(dla, w, v[8]);
                }
                Tr[i] = __fmul_rn(Tr[i], __fsub_rn(1.f, a));
            }
            warp_reduce_scatter16(v, lane);
            if ((lane & 1) == 0 && (lane >> 1) < 9) s_red[j][warp][lane >> 1] = v[0];
        }
        __syncthreads();
        for (int i = tid; i < n * 9; i += NT) {
            const int j = i / 9, q = i % 9;
            float s = 0.f;
#pragma unroll
            for (int w = 0; w < NW; ++w) s += s_red[j][w][q];
            const int64_t ei = s_e[j];
            if (ei >= 0) {
                if (q < 8)
                    partial[8 * ei + q] = s;
                else
                    partial_o[ei] = s;
            }
        }
        __syncthreads();
    }
    // Entries past every pixel's stop contribute nothing: zero their sums.
    for (int k = tg.b + nmax + tid; k < tg.e; k += NT) {
        const uint32_t g = ids[k];
        if (!gi_in_bounds(g < (uint32_t)B.total_gauss, status)) continue;
        const int64_t ei = emission_index(rect, pair_off, g, tg.tx, tg.ty, capacity);
        if (ei >= 0) {
            reinterpret_cast<float4*>(partial)[2 * ei] = make_float4(0.f, 0.f, 0.f, 0.f);
            reinterpret_cast<float4*>(partial)[2 * ei + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
            partial_o[ei] = 0.f;
        }
    }
}

}  // namespace

cudaError_t launch_render_blend(const float4* rec_binned, const uint32_t* ids, const int2* ranges, const Batch& B,
                                const float* target, float* out, float* dl_tiled, double* loss_sum, uint32_t* status,
                                cudaStream_t s) {
    if (B.total_tiles <= 0) return cudaSuccess;
    if (B.tile != kBT) return cudaErrorInvalidValue;
    return launch_pdl(k_render_blend<kBlendRenderPx>, dim3(B.total_tiles), dim3(kBPix / kBlendRenderPx), 0, s,
                      rec_binned, ids, B.opac.o, ranges, B, target, out, B.opac.n_last, dl_tiled, loss_sum, status);
}

cudaError_t launch_backward_blend(const float4* rec_binned, const uint32_t* ids, const int2* ranges, const int4* rect,
                                  const int64_t* pair_off, const Batch& B, const float* out, const float* dl_tiled,
                                  int64_t capacity, float4* partial, uint32_t* status, cudaStream_t s) {
    if (B.total_tiles <= 0) return cudaSuccess;
    if (B.tile != kBT) return cudaErrorInvalidValue;
    return launch_pdl(k_backward_blend<kBlendBackwardPx>, dim3(B.total_tiles), dim3(kBPix / kBlendBackwardPx), 0, s,
                      rec_binned, ids, B.opac.o, ranges, rect, pair_off, B, out, B.opac.n_last, dl_tiled, capacity,
                      reinterpret_cast<float*>(partial), B.opac.partial, status);
}

}  // namespace gi
