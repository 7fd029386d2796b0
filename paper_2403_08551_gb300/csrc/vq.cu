// vq.cu -- codec decode (Sec. 3.3): FP16 positions, and Cholesky / colour
// attributes as the sum over M residual-VQ stages of codebook rows,
//   hat c^M = sum_{k=1..M} C^k[i^k].
// The result equals the sum evaluated exactly and rounded once to FP32: for
// M <= 2 a single FP32 addition already is that (rounding a double-precision
// sum of two floats to float is innocuous since 53 >= 2*24 + 2); for M > 2
// the stages are accumulated in FP64 and rounded once.
#include <algorithm>

#include <cuda_fp16.h>

#include "kernels.cuh"

namespace gi {
namespace {

__global__ void __launch_bounds__(256) k_vq_decode(const uint16_t* __restrict__ means16,
                                                   const uint8_t* __restrict__ idx, const float* __restrict__ cb,
                                                   int n, int stages, int cbs, float* __restrict__ means,
                                                   float* __restrict__ chol, float* __restrict__ color,
                                                   int aos_stride, uint32_t* status) {
    extern __shared__ float scb[];  // [2][stages][cbs][3]
    const int ncb = 2 * stages * cbs * 3;
    for (int i = threadIdx.x; i < ncb; i += blockDim.x) scb[i] = cb[i];
    __syncthreads();
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
        const float mx = __half2float(__ushort_as_half(means16[2 * (size_t)g]));
        const float my = __half2float(__ushort_as_half(means16[2 * (size_t)g + 1]));
        float o[2][3];
        for (int a = 0; a < 2; ++a) {
            if (stages <= 2) {
                float acc[3] = {0.f, 0.f, 0.f};
                for (int s = 0; s < stages; ++s) {
                    int i = idx[((size_t)a * stages + s) * n + g];
                    if (i >= cbs) {  // index outside the codebook: skip the read
                        flag_error(status, kErrBounds);
                        i = 0;
                    }
                    const float* row = scb + (((size_t)a * stages + s) * cbs + i) * 3;
                    acc[0] = __fadd_rn(acc[0], row[0]);
                    acc[1] = __fadd_rn(acc[1], row[1]);
                    acc[2] = __fadd_rn(acc[2], row[2]);
                }
                o[a][0] = acc[0]; o[a][1] = acc[1]; o[a][2] = acc[2];
            } else {
                double acc[3] = {0.0, 0.0, 0.0};
                for (int s = 0; s < stages; ++s) {
                    int i = idx[((size_t)a * stages + s) * n + g];
                    if (i >= cbs) {
                        flag_error(status, kErrBounds);
                        i = 0;
                    }
                    const float* row = scb + (((size_t)a * stages + s) * cbs + i) * 3;
                    acc[0] += (double)row[0];
                    acc[1] += (double)row[1];
                    acc[2] += (double)row[2];
                }
                o[a][0] = (float)acc[0]; o[a][1] = (float)acc[1]; o[a][2] = (float)acc[2];
            }
        }
        if (aos_stride == 8) {
            float4* p = reinterpret_cast<float4*>(means) + 2 * (size_t)g;
            p[0] = make_float4(mx, my, o[0][0], o[0][1]);
            p[1] = make_float4(o[0][2], o[1][0], o[1][1], o[1][2]);
        } else {
            means[2 * (size_t)g] = mx;
            means[2 * (size_t)g + 1] = my;
            chol[3 * (size_t)g] = o[0][0];
            chol[3 * (size_t)g + 1] = o[0][1];
            chol[3 * (size_t)g + 2] = o[0][2];
            color[3 * (size_t)g] = o[1][0];
            color[3 * (size_t)g + 1] = o[1][1];
            color[3 * (size_t)g + 2] = o[1][2];
        }
    }
}

// One quad of the fast path below (at most two stages): the four
// Gaussians' attributes from their index words w[attribute][stage] and the
// padded codebook rows, then the 16-byte stores.
__device__ __forceinline__ void vq_store_quad(int q, uint4 h, const uint32_t (&w)[2][2], const float4* srow,
                                              int stages, int cbs, float4* __restrict__ means,
                                              float4* __restrict__ chol, float4* __restrict__ color,
                                              uint32_t* status) {
    float o[2][4][3];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
#pragma unroll
        for (int j = 0; j < 4; ++j) o[a][j][0] = o[a][j][1] = o[a][j][2] = 0.f;
#pragma unroll
        for (int st = 0; st < 2; ++st) {
            if (st < stages) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    int i = (w[a][st] >> (8 * j)) & 0xff;
                    if (i >= cbs) {  // index outside the codebook: skip the read
                        flag_error(status, kErrBounds);
                        i = 0;
                    }
                    const float4 r = srow[((size_t)a * stages + st) * cbs + i];
                    o[a][j][0] = __fadd_rn(o[a][j][0], r.x);
                    o[a][j][1] = __fadd_rn(o[a][j][1], r.y);
                    o[a][j][2] = __fadd_rn(o[a][j][2], r.z);
                }
            }
        }
    }
    const uint32_t hw[4] = {h.x, h.y, h.z, h.w};
    float mf[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        mf[2 * j] = __half2float(__ushort_as_half((unsigned short)(hw[j] & 0xffffu)));
        mf[2 * j + 1] = __half2float(__ushort_as_half((unsigned short)(hw[j] >> 16)));
    }
    means[2 * (size_t)q] = make_float4(mf[0], mf[1], mf[2], mf[3]);
    means[2 * (size_t)q + 1] = make_float4(mf[4], mf[5], mf[6], mf[7]);
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        float4* dst = (a == 0 ? chol : color) + 3 * (size_t)q;
        dst[0] = make_float4(o[a][0][0], o[a][0][1], o[a][0][2], o[a][1][0]);
        dst[1] = make_float4(o[a][1][1], o[a][1][2], o[a][2][0], o[a][2][1]);
        dst[2] = make_float4(o[a][2][2], o[a][3][0], o[a][3][1], o[a][3][2]);
    }
}

constexpr int kVqQuads = 2;  // quads per thread and round of the fast path (4 measured slower)

// Four consecutive Gaussians per thread when every array is 16-byte aligned
// (the usual case): the FP16 positions of the four as one 16-byte load, each
// index plane as one 4-byte load, codebook rows from shared memory as one
// 16-byte load each (rows padded to four floats), and the outputs as whole
// 16-byte stores (2 for the positions, 3 for each attribute). Same
// arithmetic as k_vq_decode.
__global__ void __launch_bounds__(256) k_vq_decode4(const uint2* __restrict__ means16, const uint8_t* __restrict__ idx,
                                                    const float* __restrict__ cb, int n, int stages, int cbs,
                                                    float4* __restrict__ means, float4* __restrict__ chol,
                                                    float4* __restrict__ color, uint32_t* status) {
    extern __shared__ float4 srow[];  // [2][stages][cbs] rows (x, y, z, 0)
    const int nrow = 2 * stages * cbs;
    for (int i = threadIdx.x; i < nrow; i += blockDim.x)
        srow[i] = make_float4(cb[3 * i], cb[3 * i + 1], cb[3 * i + 2], 0.f);
    __syncthreads();
    const int nq = n >> 2;  // whole quads; the tail is left to k_vq_decode
    const int stride = gridDim.x * blockDim.x;
    if (stages <= 2) {
        // kVqQuads quads per round, every load of the round issued before any
        // quad is decoded (the loads' latency overlaps)
        const uint4* M = reinterpret_cast<const uint4*>(means16);
        for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += kVqQuads * stride) {
            uint4 h[kVqQuads];
            uint32_t w[kVqQuads][2][2];
#pragma unroll
            for (int u = 0; u < kVqQuads; ++u) {
                const int qu = q + u * stride;
                const bool in = qu < nq;
                h[u] = in ? M[qu] : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int st = 0; st < 2; ++st) {
                        const uint32_t* I = reinterpret_cast<const uint32_t*>(idx + ((size_t)a * stages + st) * n);
                        w[u][a][st] = st < stages && in ? I[qu] : 0u;
                    }
            }
#pragma unroll
            for (int u = 0; u < kVqQuads; ++u)
                if (q + u * stride < nq)
                    vq_store_quad(q + u * stride, h[u], w[u], srow, stages, cbs, means, chol, color, status);
        }
        return;
    }
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += stride) {
        const uint4 h = reinterpret_cast<const uint4*>(means16)[q];  // 4 Gaussians x (x, y) binary16
        float o[2][4][3];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            if (stages <= 2) {
#pragma unroll
                for (int j = 0; j < 4; ++j) o[a][j][0] = o[a][j][1] = o[a][j][2] = 0.f;
                for (int s = 0; s < stages; ++s) {
                    const uint32_t w = reinterpret_cast<const uint32_t*>(idx + ((size_t)a * stages + s) * n)[q];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        int i = (w >> (8 * j)) & 0xff;
                        if (i >= cbs) {  // index outside the codebook: skip the read
                            flag_error(status, kErrBounds);
                            i = 0;
                        }
                        const float4 r = srow[((size_t)a * stages + s) * cbs + i];
                        o[a][j][0] = __fadd_rn(o[a][j][0], r.x);
                        o[a][j][1] = __fadd_rn(o[a][j][1], r.y);
                        o[a][j][2] = __fadd_rn(o[a][j][2], r.z);
                    }
                }
            } else {
                double acc[4][3] = {};
                for (int s = 0; s < stages; ++s) {
                    const uint32_t w = reinterpret_cast<const uint32_t*>(idx + ((size_t)a * stages + s) * n)[q];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        int i = (w >> (8 * j)) & 0xff;
                        if (i >= cbs) {
                            flag_error(status, kErrBounds);
                            i = 0;
                        }
                        const float4 r = srow[((size_t)a * stages + s) * cbs + i];
                        acc[j][0] += (double)r.x;
                        acc[j][1] += (double)r.y;
                        acc[j][2] += (double)r.z;
                    }
                }
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    for (int c = 0; c < 3; ++c) o[a][j][c] = (float)acc[j][c];
            }
        }
        const uint32_t hw[4] = {h.x, h.y, h.z, h.w};
        float mf[8];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            mf[2 * j] = __half2float(__ushort_as_half((unsigned short)(hw[j] & 0xffffu)));
            mf[2 * j + 1] = __half2float(__ushort_as_half((unsigned short)(hw[j] >> 16)));
        }
        means[2 * (size_t)q] = make_float4(mf[0], mf[1], mf[2], mf[3]);
        means[2 * (size_t)q + 1] = make_float4(mf[4], mf[5], mf[6], mf[7]);
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            float4* dst = (a == 0 ? chol : color) + 3 * (size_t)q;
            dst[0] = make_float4(o[a][0][0], o[a][0][1], o[a][0][2], o[a][1][0]);
            dst[1] = make_float4(o[a][1][1], o[a][1][2], o[a][2][0], o[a][2][1]);
            dst[2] = make_float4(o[a][2][2], o[a][3][0], o[a][3][1], o[a][3][2]);
        }
    }
}

// The paper's codec (Sec. 3.3): FP16 positions, the b-bit Cholesky codes
// reconstructed as l_bar_i = code_i gamma_i + beta_i (Eq. 9, the same two
// roundings as the fit's quantiser), and the RVQ colour as the FP64 sum of
// the chosen entries in stage order, rounded once (as the fit's formation).
__global__ void __launch_bounds__(256) k_codec_decode(const uint16_t* __restrict__ means16,
                                                      const uchar4* __restrict__ codes, GammaBeta gb,
                                                      const uint8_t* __restrict__ idx, const float* __restrict__ cb,
                                                      int n, int stages, int size, float* __restrict__ means,
                                                      float* __restrict__ chol, float* __restrict__ color,
                                                      uint32_t* status) {
    extern __shared__ float scb[];  // [stages][size][3]
    for (int i = threadIdx.x; i < stages * size * 3; i += blockDim.x) scb[i] = cb[i];
    __syncthreads();
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
        means[2 * (size_t)g] = __half2float(__ushort_as_half(means16[2 * (size_t)g]));
        means[2 * (size_t)g + 1] = __half2float(__ushort_as_half(means16[2 * (size_t)g + 1]));
        const uchar4 q = codes[g];
        chol[3 * (size_t)g] = __fadd_rn(__fmul_rn((float)q.x, gb.v[0]), gb.v[3]);
        chol[3 * (size_t)g + 1] = __fadd_rn(__fmul_rn((float)q.y, gb.v[1]), gb.v[4]);
        chol[3 * (size_t)g + 2] = __fadd_rn(__fmul_rn((float)q.z, gb.v[2]), gb.v[5]);
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int m = 0; m < stages; ++m) {
            int j = idx[(size_t)m * n + g];
            if (j >= size) {  // index outside the codebook: skip the read
                flag_error(status, kErrBounds);
                j = 0;
            }
            const float* e = scb + ((size_t)m * size + j) * 3;
            s0 = __dadd_rn(s0, (double)e[0]);
            s1 = __dadd_rn(s1, (double)e[1]);
            s2 = __dadd_rn(s2, (double)e[2]);
        }
        color[3 * (size_t)g] = (float)s0;
        color[3 * (size_t)g + 1] = (float)s1;
        color[3 * (size_t)g + 2] = (float)s2;
    }
}

}  // namespace

cudaError_t launch_codec_decode(const uint16_t* means16, const uint8_t* codes, const float* gamma_beta,
                                const uint8_t* idx, const float* cb, int32_t n, int32_t stages, int32_t size,
                                float* means, float* chol, float* color, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    GammaBeta gb;
    for (int i = 0; i < 6; ++i) gb.v[i] = gamma_beta[i];
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 148;
    const int blocks = std::max(1, std::min((n + 255) / 256, nsm * 4));
    k_codec_decode<<<blocks, 256, (size_t)stages * size * 3 * sizeof(float), s>>>(
        means16, reinterpret_cast<const uchar4*>(codes), gb, idx, cb, n, stages, size, means, chol, color,
        device_status());
    return cudaGetLastError();
}

cudaError_t launch_vq_decode(const uint16_t* means16, const uint8_t* idx, const float* cb, int32_t n, int32_t stages,
                             int32_t cb_size, float* means, float* chol, float* color, int32_t out_stride_aos,
                             cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    auto a16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    if (out_stride_aos == 0 && n % 4 == 0 && a16(means16) && (reinterpret_cast<uintptr_t>(idx) & 3) == 0 &&
        a16(means) && a16(chol) && a16(color)) {
        const size_t smem = (size_t)2 * stages * cb_size * sizeof(float4);
        cudaError_t e = smem_optin(reinterpret_cast<const void*>(k_vq_decode4), (int)smem);
        if (e != cudaSuccess) return e;
        const int blocks = std::max(1, std::min((n / 4 + 255) / 256, sm_count() * 8));
        k_vq_decode4<<<blocks, 256, smem, s>>>(reinterpret_cast<const uint2*>(means16), idx, cb, n, stages, cb_size,
                                               reinterpret_cast<float4*>(means), reinterpret_cast<float4*>(chol),
                                               reinterpret_cast<float4*>(color), device_status());
        return cudaGetLastError();
    }
    const size_t smem = (size_t)2 * stages * cb_size * 3 * sizeof(float);
    {
        cudaError_t e = smem_optin(reinterpret_cast<const void*>(k_vq_decode), (int)smem);
        if (e != cudaSuccess) return e;
    }
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 148;
    const int blocks = std::max(1, std::min((n + 255) / 256, nsm * 4));
    k_vq_decode<<<blocks, 256, smem, s>>>(means16, idx, cb, n, stages, cb_size, means, chol, color, out_stride_aos,
                                          device_status());
    return cudaGetLastError();
}

}  // namespace gi
