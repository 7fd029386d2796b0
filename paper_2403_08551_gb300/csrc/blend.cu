// blend.cu -- sorted alpha-blending render and its gradients (Sec. 3.2,
// Eq. 3-4): the rasterisation that accumulated summation replaces, built to
// measure that replacement on the same hardware (Table 3's "w/o AR").
//
//   alpha_n = min(0.99, o_n exp(-sigma_n)), skipped when alpha_n < 1/255,
//   C_i = sum_n c_n alpha_n T_n, T_n = prod_{m < n} (1 - alpha_m),
//   the walk stopping before the Gaussian that would take T below 1e-4
//
// over each tile's list in ascending Gaussian index (a 2D image has no depth
// to sort by). One CTA per 16 x 16 tile, one thread per pixel: the list is
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
// are summed over the tile's 256 pixels (warp butterflies, then the warps in
// order) into the same eight per-pair sums the accumulated backward writes
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

__global__ void __launch_bounds__(kBPix) k_render_blend(const float4* __restrict__ rec_binned,
                                                        const uint32_t* __restrict__ ids,
                                                        const float* __restrict__ o_eff,
                                                        const int2* __restrict__ ranges, Batch B,
                                                        const float* __restrict__ target, float* __restrict__ out,
                                                        int32_t* __restrict__ n_last, float* __restrict__ dl_tiled,
                                                        double* __restrict__ loss_sum, uint32_t* status) {
    __shared__ float4 s_rec[kBPix][2];
    __shared__ float s_o[kBPix];
    __shared__ float s_red[kBWarps];
    pdl_wait();
    const int t = blockIdx.x;
    const TileGeo tg = tile_geo(B, ranges, t, status);
    const ImgDesc& d = tg.d;
    const int p = threadIdx.x;
    const int x = tg.tx * kBT + p % kBT, y = tg.ty * kBT + p / kBT;
    const bool inside = x < d.W && y < d.H;
    const float px = (float)x + 0.5f, py = (float)y + 0.5f;
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, Tr = 1.f;
    int last = 0;
    bool done = !inside;
    for (int base = tg.b; base < tg.e; base += kBPix) {
        if (__syncthreads_and(done)) break;  // also orders the restaging after the last chunk's reads
        const int k = base + p;
        if (k < tg.e) {
            uint32_t g = ids[k];
            if (!gi_in_bounds(g < (uint32_t)B.total_gauss, status)) g = 0;
            s_rec[p][0] = rec_binned[2 * (size_t)k];
            s_rec[p][1] = rec_binned[2 * (size_t)k + 1];
            s_o[p] = o_eff[g];
        }
        __syncthreads();
        const int n = min(kBPix, tg.e - base);
        if (!done) {
            for (int j = 0; j < n; ++j) {
                float dx, dy;
                const float4 r1 = s_rec[j][1];
                const float w = blend_w(s_rec[j][0], r1, px, py, dx, dy);
                float a = __fmul_rn(s_o[j], w);
                if (a < kBlendAlphaMin) continue;
                a = fminf(a, kBlendAlphaMax);
                const float test = __fmul_rn(Tr, __fsub_rn(1.f, a));
                if (test < kBlendTMin) {
                    done = true;
                    break;
                }
                const float at = __fmul_rn(a, Tr);
                C0 = __fadd_rn(C0, __fmul_rn(r1.y, at));
                C1 = __fadd_rn(C1, __fmul_rn(r1.z, at));
                C2 = __fadd_rn(C2, __fmul_rn(r1.w, at));
                Tr = test;
                last = base - tg.b + j + 1;
            }
        }
    }
    const float scale = 2.0f / (3.0f * (float)d.W * (float)d.H);
    float dl0 = 0.f, dl1 = 0.f, dl2 = 0.f, lsum = 0.f;
    if (inside) {
        const int64_t pix = d.pix_base + (int64_t)y * d.W + x;
        out[3 * pix] = C0;
        out[3 * pix + 1] = C1;
        out[3 * pix + 2] = C2;
        if (n_last) n_last[pix] = last;
        if (target) {
            const float r0 = C0 - target[3 * pix], r1 = C1 - target[3 * pix + 1], r2 = C2 - target[3 * pix + 2];
            lsum = fmaf(r2, r2, fmaf(r1, r1, r0 * r0));
            dl0 = r0 * scale;
            dl1 = r1 * scale;
            dl2 = r2 * scale;
        }
    }
    if (dl_tiled) {  // planar per tile, as the accumulated render writes it
        float* dt = dl_tiled + (size_t)t * 3 * kBPix;
        dt[p] = dl0;
        dt[kBPix + p] = dl1;
        dt[2 * kBPix + p] = dl2;
    }
    if (target && loss_sum) {
        lsum = warp_sum(lsum);
        if ((p & 31) == 0) s_red[p >> 5] = lsum;
        __syncthreads();
        if (p == 0) {
            float s = 0.f;
            for (int w = 0; w < kBWarps; ++w) s += s_red[w];
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

__global__ void __launch_bounds__(kBPix) k_backward_blend(
    const float4* __restrict__ rec_binned, const uint32_t* __restrict__ ids, const float* __restrict__ o_eff,
    const int2* __restrict__ ranges, const int4* __restrict__ rect, const int64_t* __restrict__ pair_off, Batch B,
    const float* __restrict__ out, const int32_t* __restrict__ n_last, const float* __restrict__ dl_tiled,
    int64_t capacity, float* __restrict__ partial, float* __restrict__ partial_o, uint32_t* status) {
    __shared__ float4 s_rec[kBChunk][2];
    __shared__ float s_o[kBChunk];
    __shared__ int64_t s_e[kBChunk];
    __shared__ float s_red[kBChunk][kBWarps][9];
    __shared__ int s_max[kBWarps];
    pdl_wait();
    const int t = blockIdx.x;
    const TileGeo tg = tile_geo(B, ranges, t, status);
    const ImgDesc& d = tg.d;
    const int p = threadIdx.x, lane = p & 31, warp = p >> 5;
    const int x = tg.tx * kBT + p % kBT, y = tg.ty * kBT + p / kBT;
    const bool inside = x < d.W && y < d.H;
    const float px = (float)x + 0.5f, py = (float)y + 0.5f;
    const float* dt = dl_tiled + (size_t)t * 3 * kBPix;
    const float g0 = dt[p], g1 = dt[kBPix + p], g2 = dt[2 * kBPix + p];
    float Cf0 = 0.f, Cf1 = 0.f, Cf2 = 0.f;
    int nl = 0;
    if (inside) {
        const int64_t pix = d.pix_base + (int64_t)y * d.W + x;
        Cf0 = out[3 * pix];
        Cf1 = out[3 * pix + 1];
        Cf2 = out[3 * pix + 2];
        nl = min(n_last[pix], tg.e - tg.b);
    }
    {
        const int m = __reduce_max_sync(0xffffffffu, nl);
        if (lane == 0) s_max[warp] = m;
    }
    __syncthreads();
    int nmax = 0;
#pragma unroll
    for (int w = 0; w < kBWarps; ++w) nmax = max(nmax, s_max[w]);
    float P0 = 0.f, P1 = 0.f, P2 = 0.f, Tr = 1.f;
    for (int base = tg.b; base < tg.b + nmax; base += kBChunk) {
        const int n = min(kBChunk, tg.b + nmax - base);
        if (p < n) {
            const int k = base + p;
            uint32_t g = ids[k];
            const bool ok = gi_in_bounds(g < (uint32_t)B.total_gauss, status);
            if (!ok) g = 0;
            s_rec[p][0] = rec_binned[2 * (size_t)k];
            s_rec[p][1] = rec_binned[2 * (size_t)k + 1];
            s_o[p] = o_eff[g];
            s_e[p] = ok ? emission_index(rect, pair_off, g, tg.tx, tg.ty, capacity) : -1;
        }
        __syncthreads();
        for (int j = 0; j < n; ++j) {
            float v[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (base - tg.b + j < nl) {
                float dx, dy;
                const float4 r1 = s_rec[j][1];
                const float w = blend_w(s_rec[j][0], r1, px, py, dx, dy);
                float a = __fmul_rn(s_o[j], w);
                if (a >= kBlendAlphaMin) {
                    const bool clamped = a > kBlendAlphaMax;
                    a = fminf(a, kBlendAlphaMax);
                    const float at = __fmul_rn(a, Tr);
                    P0 = __fadd_rn(P0, __fmul_rn(r1.y, at));
                    P1 = __fadd_rn(P1, __fmul_rn(r1.z, at));
                    P2 = __fadd_rn(P2, __fmul_rn(r1.w, at));
                    const float inv = 1.f / (1.f - a);
                    const float dla = g0 * (r1.y * Tr - (Cf0 - P0) * inv) + g1 * (r1.z * Tr - (Cf1 - P1) * inv) +
                                      g2 * (r1.w * Tr - (Cf2 - P2) * inv);
                    v[0] = g0 * at;
                    v[1] = g1 * at;
                    v[2] = g2 * at;
                    if (!clamped) {
                        const float ee = dla * a;  // -dL/dsigma
                        const float ex = ee * dx;
                        v[3] = ex;
                        v[4] = ee * dy;
                        v[5] = ex * dx;
                        v[6] = ex * dy;
                        v[7] = ee * dy * dy;
                        v[8] = dla * w;
                    }
                    Tr = __fmul_rn(Tr, __fsub_rn(1.f, a));
                }
            }
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const float s = warp_sum(v[q]);
                if (lane == 0) s_red[j][warp][q] = s;
            }
        }
        __syncthreads();
        for (int i = p; i < n * 9; i += kBPix) {
            const int j = i / 9, q = i % 9;
            float s = 0.f;
#pragma unroll
            for (int w = 0; w < kBWarps; ++w) s += s_red[j][w][q];
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
    for (int k = tg.b + nmax + p; k < tg.e; k += kBPix) {
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
    return launch_pdl(k_render_blend, dim3(B.total_tiles), dim3(kBPix), 0, s, rec_binned, ids, B.opac.o, ranges, B,
                      target, out, B.opac.n_last, dl_tiled, loss_sum, status);
}

cudaError_t launch_backward_blend(const float4* rec_binned, const uint32_t* ids, const int2* ranges, const int4* rect,
                                  const int64_t* pair_off, const Batch& B, const float* out, const float* dl_tiled,
                                  int64_t capacity, float4* partial, uint32_t* status, cudaStream_t s) {
    if (B.total_tiles <= 0) return cudaSuccess;
    if (B.tile != kBT) return cudaErrorInvalidValue;
    return launch_pdl(k_backward_blend, dim3(B.total_tiles), dim3(kBPix), 0, s, rec_binned, ids, B.opac.o, ranges,
                      rect, pair_off, B, out, B.opac.n_last, dl_tiled, capacity, reinterpret_cast<float*>(partial),
                      B.opac.partial, status);
}

}  // namespace gi
