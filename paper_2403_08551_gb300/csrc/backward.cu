// backward.cu -- gradients of the accumulated-summation render (App. A).
//
// Pass 1 (k_backward): one lane per (tile, Gaussian) pair. The lane walks
// every pixel of its tile, recomputing w = exp(-sigma) (no per-pixel state is
// kept from the forward pass) and accumulates eight sums for its pair:
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

template <int T>
__global__ void __launch_bounds__(256) k_backward(const float4* __restrict__ rec_binned,
                                                  const uint32_t* __restrict__ keys,
                                                  const uint32_t* __restrict__ ids, const int4* __restrict__ rect,
                                                  const int64_t* __restrict__ pair_off,
                                                  const float4* __restrict__ dl_tiled, Batch B,
                                                  const int64_t* __restrict__ k_dev, int64_t capacity,
                                                  float4* __restrict__ partial) {
    constexpr int NPIX = T * T;
    const int K = (int)min(*k_dev, capacity);
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int task = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; task * 32 < K; task += nwarps) {
        int k = task * 32 + lane;
        const bool valid = k < K;
        if (!valid) k = K - 1;
        const float4 r0 = rec_binned[2 * (size_t)k];      // mx, my, A', B'
        const float4 r1 = rec_binned[2 * (size_t)k + 1];  // C', c'r, c'g, c'b
        const uint32_t t = keys[k];
        const ImgDesc d = img_desc(B, image_of_tile(B, (int)t));
        const int lt = (int)t - d.tile_base;
        const int tx = lt % d.tw, ty = lt / d.tw;
        const float4* __restrict__ G = dl_tiled + (size_t)t * NPIX;
        const float dx0 = (float)(tx * T) + 0.5f - r0.x;
        const float dyb = (float)(ty * T) + 0.5f - r0.y;
        float gcr = 0.f, gcg = 0.f, gcb = 0.f;
        // Moment sums with Kahan compensation across rows: the per-pair sums
        // cancel strongly for Gaussians near equilibrium, and the row
        // partials are the large terms of that cancellation.
        float Sx = 0.f, Sy = 0.f, Sxx = 0.f, Sxy = 0.f, Syy = 0.f;
        float cSx = 0.f, cSy = 0.f, cSxx = 0.f, cSxy = 0.f, cSyy = 0.f;
#pragma unroll 1
        for (int y = 0; y < T; ++y) {
            const float dy = dyb + (float)y;
            const float bdy = r0.w * dy;
            const float cdy2 = r1.x * dy * dy;
            float u = 0.f, v = 0.f, q = 0.f;
#pragma unroll
            for (int x = 0; x < T; ++x) {
                const float4 g = __ldg(G + y * T + x);
                const float dx = dx0 + (float)x;
                const float s = fmaf(fmaf(r0.z, dx, bdy), dx, cdy2);
                const float w = ex2(-s);
                gcr = fmaf(g.x, w, gcr);
                gcg = fmaf(g.y, w, gcg);
                gcb = fmaf(g.z, w, gcb);
                const float gw = fmaf(g.z, r1.w, fmaf(g.y, r1.z, g.x * r1.y));
                const float e = gw * w;
                u += e;
                const float t1 = e * dx;
                v += t1;
                q = fmaf(t1, dx, q);
            }
            kahan_add(Sx, cSx, v);
            kahan_add(Sy, cSy, u * dy);
            kahan_add(Sxx, cSxx, q);
            kahan_add(Sxy, cSxy, v * dy);
            kahan_add(Syy, cSyy, u * dy * dy);
        }
        Sx -= cSx;
        Sy -= cSy;
        Sxx -= cSxx;
        Sxy -= cSxy;
        Syy -= cSyy;
        if (valid) {
            const uint32_t g = ids[k];
            const int4 r = rect[g];
            const int64_t p = pair_off[g] + (int64_t)(ty - r.y) * (r.z - r.x) + (tx - r.x);
            if (p >= 0 && p < capacity) {
                partial[2 * p] = make_float4(gcr, gcg, gcb, Sx);
                partial[2 * p + 1] = make_float4(Sy, Sxx, Sxy, Syy);
            }
        }
    }
}

// HWC dL/dC -> tiled float4 layout, zero outside the image.
template <int T>
__global__ void k_pack_dl(const float* __restrict__ dl, Batch B, float4* __restrict__ out) {
    const int t = blockIdx.x;
    const ImgDesc d = img_desc(B, image_of_tile(B, t));
    const int lt = t - d.tile_base;
    const int tx = lt % d.tw, ty = lt / d.tw;
    for (int p = threadIdx.x; p < T * T; p += blockDim.x) {
        const int x = tx * T + p % T, y = ty * T + p / T;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (x < d.W && y < d.H) {
            const int64_t pix = d.pix_base + (int64_t)y * d.W + x;
            v = make_float4(dl[3 * pix], dl[3 * pix + 1], dl[3 * pix + 2], 0.f);
        }
        out[(size_t)t * T * T + p] = v;
    }
}

template <bool ADAM>
__global__ void __launch_bounds__(256) k_reduce(const float4* __restrict__ partial,
                                                const int64_t* __restrict__ pair_off,
                                                const int32_t* __restrict__ cnt, int64_t capacity, int n,
                                                ParamsIn P, float* __restrict__ g_means, float* __restrict__ g_chol,
                                                float* __restrict__ g_color, float* __restrict__ g_conic,
                                                AdamCfg cfg, float* __restrict__ params, float* __restrict__ m,
                                                float* __restrict__ v, float* __restrict__ grads_aos) {
    __shared__ int s_step;
    if (ADAM) {
        if (threadIdx.x == 0) s_step = *cfg.step + 1;
        __syncthreads();
    }
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n) {
        float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        float ca[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const int c = cnt[g];
        const int64_t p0 = pair_off[g];
        const int64_t p1 = min(p0 + (int64_t)c, capacity);
        for (int64_t p = p0; p < p1; ++p) {  // emission order, compensated
            const float4 x = partial[2 * p], y = partial[2 * p + 1];
            kahan_add(a[0], ca[0], x.x); kahan_add(a[1], ca[1], x.y);
            kahan_add(a[2], ca[2], x.z); kahan_add(a[3], ca[3], x.w);
            kahan_add(a[4], ca[4], y.x); kahan_add(a[5], ca[5], y.y);
            kahan_add(a[6], ca[6], y.z); kahan_add(a[7], ca[7], y.w);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] -= ca[j];
        const float l1 = P.chol[(int64_t)g * P.ls], l2 = P.chol[(int64_t)g * P.ls + 1],
                    l3 = P.chol[(int64_t)g * P.ls + 2];
        float gr[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        float gq[3] = {0.f, 0.f, 0.f};
        if (c > 0) {
            const float s11 = l1 * l1, s12 = l1 * l2, s22 = l2 * l2 + l3 * l3;
            const float dd = l1 * l3, det = dd * dd;
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
            gr[2] = 2.f * (g1 * l1 + g2 * l2);
            gr[3] = 2.f * (g2 * l1 + g3 * l2);
            gr[4] = 2.f * g3 * l3;
            gr[5] = a[0]; gr[6] = a[1]; gr[7] = a[2];
        }
        if (!ADAM) {
            if (g_means) { g_means[2 * g] = gr[0]; g_means[2 * g + 1] = gr[1]; }
            if (g_chol) { g_chol[3 * g] = gr[2]; g_chol[3 * g + 1] = gr[3]; g_chol[3 * g + 2] = gr[4]; }
            if (g_color) { g_color[3 * g] = gr[5]; g_color[3 * g + 1] = gr[6]; g_color[3 * g + 2] = gr[7]; }
            if (g_conic) { g_conic[3 * g] = gq[0]; g_conic[3 * g + 1] = gq[1]; g_conic[3 * g + 2] = gq[2]; }
        } else {
            if (grads_aos) {
                float4* go = reinterpret_cast<float4*>(grads_aos) + 2 * (size_t)g;
                go[0] = make_float4(gr[0], gr[1], gr[2], gr[3]);
                go[1] = make_float4(gr[4], gr[5], gr[6], gr[7]);
            }
            const int step = s_step;
            const float bc1 = 1.f - powf(cfg.beta1, (float)step);
            const float bc2 = 1.f - powf(cfg.beta2, (float)step);
            const float rs2 = rsqrtf(bc2);
            float4* P4 = reinterpret_cast<float4*>(params) + 2 * (size_t)g;
            float4* M4 = reinterpret_cast<float4*>(m) + 2 * (size_t)g;
            float4* V4 = reinterpret_cast<float4*>(v) + 2 * (size_t)g;
            float pp[8], mm[8], vv[8];
            *reinterpret_cast<float4*>(pp) = P4[0]; *reinterpret_cast<float4*>(pp + 4) = P4[1];
            *reinterpret_cast<float4*>(mm) = M4[0]; *reinterpret_cast<float4*>(mm + 4) = M4[1];
            *reinterpret_cast<float4*>(vv) = V4[0]; *reinterpret_cast<float4*>(vv + 4) = V4[1];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float lr = cfg.lr[j < 2 ? 0 : (j < 5 ? 1 : 2)];
                mm[j] = cfg.beta1 * mm[j] + (1.f - cfg.beta1) * gr[j];
                vv[j] = cfg.beta2 * vv[j] + (1.f - cfg.beta2) * gr[j] * gr[j];
                const float denom = sqrtf(vv[j]) * rs2 + cfg.eps;
                pp[j] -= (lr / bc1) * mm[j] / denom;
            }
            P4[0] = *reinterpret_cast<float4*>(pp); P4[1] = *reinterpret_cast<float4*>(pp + 4);
            M4[0] = *reinterpret_cast<float4*>(mm); M4[1] = *reinterpret_cast<float4*>(mm + 4);
            V4[0] = *reinterpret_cast<float4*>(vv); V4[1] = *reinterpret_cast<float4*>(vv + 4);
        }
    }
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

int sm_count_b() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
    return v;
}

}  // namespace

cudaError_t launch_backward(const float4* rec_binned, const uint32_t* keys, const uint32_t* ids, const int4* rect,
                            const int64_t* pair_off, const float4* dl_tiled, const Batch& B, const int64_t* k_dev,
                            int64_t capacity, float4* partial, cudaStream_t s) {
    if (capacity <= 0) return cudaSuccess;
    static int nsm = 0;
    if (!nsm) nsm = sm_count_b();
    const int64_t need = (capacity + 255) / 256;  // 8 warps x 32 pairs per block-iteration
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)nsm * 8));
    switch (B.tile) {
        case 8:
            k_backward<8><<<blocks, 256, 0, s>>>(rec_binned, keys, ids, rect, pair_off, dl_tiled, B, k_dev, capacity,
                                                 partial);
            break;
        case 16:
            k_backward<16><<<blocks, 256, 0, s>>>(rec_binned, keys, ids, rect, pair_off, dl_tiled, B, k_dev,
                                                  capacity, partial);
            break;
        case 32:
            k_backward<32><<<blocks, 256, 0, s>>>(rec_binned, keys, ids, rect, pair_off, dl_tiled, B, k_dev,
                                                  capacity, partial);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_pack_dl(const float* dl_hwc, const Batch& B, float4* dl_tiled, cudaStream_t s) {
    if (B.total_tiles <= 0) return cudaSuccess;
    switch (B.tile) {
        case 8: k_pack_dl<8><<<B.total_tiles, 64, 0, s>>>(dl_hwc, B, dl_tiled); break;
        case 16: k_pack_dl<16><<<B.total_tiles, 256, 0, s>>>(dl_hwc, B, dl_tiled); break;
        case 32: k_pack_dl<32><<<B.total_tiles, 256, 0, s>>>(dl_hwc, B, dl_tiled); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_reduce(const float4* partial, const int64_t* pair_off, const int32_t* cnt, int64_t capacity,
                          int32_t n, const ParamsIn& P, float* g_means, float* g_chol, float* g_color,
                          float* g_conic, const AdamCfg* adam, float* params, float* m, float* v, float* grads_aos,
                          cudaStream_t s) {
    const int blocks = std::max(1, (n + 255) / 256);
    if (adam) {
        k_reduce<true><<<blocks, 256, 0, s>>>(partial, pair_off, cnt, capacity, n, P, nullptr, nullptr, nullptr,
                                              nullptr, *adam, params, m, v, grads_aos);
    } else {
        AdamCfg none{};
        k_reduce<false><<<blocks, 256, 0, s>>>(partial, pair_off, cnt, capacity, n, P, g_means, g_chol, g_color,
                                               g_conic, none, nullptr, nullptr, nullptr, nullptr);
    }
    return cudaGetLastError();
}

}  // namespace gi
