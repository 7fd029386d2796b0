// bin.cu -- Gaussian formation (projection to conic + tile rect) and tile
// binning: count scan, key emission, stable LSD radix sort (onesweep with a
// bounded decoupled look-back) and per-tile ranges.
//
// Formation follows Sec. 3.1, Eq. 1 (Sigma = L L^T) and Sec. 3.2, Eq. 5
// (sigma = 1/2 d^T Sigma^-1 d). With Sigma^-1 = L^-T L^-1, sigma = 1/2 |L^-1 d|^2;
// the record stores the scaled inverse factor so that the kernels evaluate
// sigma as a sum of two squares, which stays accurate for needle-shaped
// Gaussians where the expanded quadratic form cancels catastrophically. The paper does not define the screen support
// of a Gaussian; the reading implemented here is the tile-granular 3-sigma
// rectangle, evaluated with correctly rounded FP32 operations only (no fused
// multiply-add), so that tile lists are bit-identical to the CPU oracle.
// Binning keeps ascending Gaussian index inside each tile (the sort is
// stable over keys emitted in Gaussian order), which fixes the summation
// order of Eq. 7 and makes the forward render reproducible.
#include <cuda_fp16.h>

#include <algorithm>

#include "kernels.cuh"

namespace gi {

namespace {

constexpr int kWin = 16;  // look-back window (predecessor words loaded at once)

__device__ __forceinline__ float clampf_(float v, float lo, float hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

// tanh in FP64 as (1 - e) / (1 + e), e = exp(-2|x|), sign restored: a few
// ulp of FP64, far below the FP32 rounding that follows, and cheaper than the
// library tanh on this part's FP64 units (the App. C.1 positions).
__device__ __forceinline__ double tanh_fp64(double x) {
    const double e = exp(-2.0 * fabs(x));
    return copysign((1.0 - e) / (1.0 + e), x);
}

__device__ void zero_job(const ZeroJob& zj) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        uint32_t* p = zj.p[r];
        if (!p) continue;
        const int64_t n = zj.n32[r], n4 = n >> 2;
        uint4* p4 = reinterpret_cast<uint4*>(p);
        for (int64_t i = tid; i < n4; i += nth) p4[i] = make_uint4(0, 0, 0, 0);
        for (int64_t i = (n4 << 2) + tid; i < n; i += nth) p[i] = 0u;
    }
}

// ---------------------------------------------------------------------------
// Formation: conic + FP32 3-sigma tile rect (Eq. 1, Eq. 5).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kProjBlock) k_project(ParamsIn P, Batch B, float4* __restrict__ rec,
                                                        int4* __restrict__ rect, int32_t* __restrict__ cnt,
                                                        int64_t* __restrict__ blk_sum, ZeroJob zj,
                                                        uint32_t* __restrict__ M, uint32_t* __restrict__ chunk_sum) {
    constexpr int CPB = kProjBlock / kCmChunk;  // count-matrix chunks per projection block
    static_assert(kProjBlock % kCmChunk == 0, "a projection block holds whole count-matrix chunks");
    extern __shared__ uint32_t s_h[];  // with M: [CPB][total_tiles] tile histograms of the block's chunks
    __shared__ int64_t s_warp[32];
    __shared__ uint32_t s_tot[CPB];
    pdl_wait();
    zero_job(zj);
    if (M) {
        for (int i = threadIdx.x; i < CPB * B.total_tiles; i += blockDim.x) s_h[i] = 0u;
        if (threadIdx.x < CPB) s_tot[threadIdx.x] = 0u;
        __syncthreads();
    }
    const int g = blockIdx.x * kProjBlock + threadIdx.x;
    int c = 0;
    if (g < B.total_gauss) {
        const ImgDesc d = img_desc(B, image_of_gauss(B, g));
        float mx = P.means[(int64_t)g * P.ms], my = P.means[(int64_t)g * P.ms + 1];
        float l1 = P.chol[(int64_t)g * P.ls], l2 = P.chol[(int64_t)g * P.ls + 1], l3 = P.chol[(int64_t)g * P.ls + 2];
        if (B.param_mode == 1) {
            // App. C.1: positions through tanh into (-1, 1), read as
            // mu = (tanh(theta) + 1) / 2 * (W, H) (tanh in FP64, one rounding
            // to FP32); +0.5 on the Cholesky diagonal or on the scales.
            mx = (float)__dmul_rn(__dmul_rn(__dadd_rn(tanh_fp64((double)mx), 1.0), 0.5), (double)d.W);
            my = (float)__dmul_rn(__dmul_rn(__dadd_rn(tanh_fp64((double)my), 1.0), 0.5), (double)d.H);
            if (B.cov_mode == 0) {
                l1 = __fadd_rn(l1, 0.5f);
                l3 = __fadd_rn(l3, 0.5f);
            }
        }
        if (B.cov_mode == 1) {
            // Rotation-scaling form (Sec. 3.1, Eq. 2-3): the slots hold
            // (theta, s1, s2); the equivalent Cholesky vector of
            // Sigma = (R S)(R S)^T, in FP64 with one rounding per entry:
            // l1 = sqrt(Sigma11), l2 = Sigma12 / l1, l3 = |s1 s2| / l1.
            const double th = (double)l1;
            double s1 = (double)l2, s2 = (double)l3;
            if (B.param_mode == 1) {
                s1 = __dadd_rn(s1, 0.5);
                s2 = __dadd_rn(s2, 0.5);
            }
            double sn, cs;
            sincos(th, &sn, &cs);
            const double S11 = __dadd_rn(__dmul_rn(__dmul_rn(__dmul_rn(cs, cs), s1), s1),
                                         __dmul_rn(__dmul_rn(__dmul_rn(sn, sn), s2), s2));
            const double S12 = __dmul_rn(__dmul_rn(cs, sn), __dsub_rn(__dmul_rn(s1, s1), __dmul_rn(s2, s2)));
            const double q1 = __dsqrt_rn(S11);
            l1 = (float)q1;
            l2 = (float)__ddiv_rn(S12, q1);
            l3 = (float)__ddiv_rn(fabs(__dmul_rn(s1, s2)), q1);
        }
        float cr = P.color[(int64_t)g * P.cs], cg = P.color[(int64_t)g * P.cs + 1],
              cb = P.color[(int64_t)g * P.cs + 2];
        if (B.opac.mode > 0) {
            // Separate opacity o = sigmoid(logit) (FP64, one rounding). With
            // accumulated summation the record carries c' = c o (Eq. 5); the
            // blending render reads o itself and the record keeps c.
            const float o = (float)__ddiv_rn(1.0, __dadd_rn(1.0, exp(-(double)B.opac.logit[g])));
            B.opac.o[g] = o;
            if (B.opac.mode == 1) {
                cr = __fmul_rn(cr, o);
                cg = __fmul_rn(cg, o);
                cb = __fmul_rn(cb, o);
            }
        }
        if (B.codec.bits > 0) {
            // Codec fine-tuning (Sec. 3.3): FP16 positions, b-bit Cholesky
            // vector, greedy RVQ colour; the codes are the encoded stream.
            const CodecCfg& Q = B.codec;
            const __half hx = __float2half_rn(mx), hy = __float2half_rn(my);
            mx = __half2float(hx);
            my = __half2float(hy);
            if (Q.means16) {
                Q.means16[2 * (size_t)g] = __half_as_ushort(hx);
                Q.means16[2 * (size_t)g + 1] = __half_as_ushort(hy);
            }
            float x, q0, q1, q2;
            l1 = lsq_quant(l1, Q.gb[0], Q.gb[3], Q.qp, x, q0);
            l2 = lsq_quant(l2, Q.gb[1], Q.gb[4], Q.qp, x, q1);
            l3 = lsq_quant(l3, Q.gb[2], Q.gb[5], Q.qp, x, q2);
            auto code8 = [](float q) { return (unsigned char)(q >= 0.f && q <= 255.f ? (int)q : 0); };
            Q.codes[g] = make_uchar4(code8(q0), code8(q1), code8(q2), 0);
            float r0 = cr, r1 = cg, r2 = cb;
            double s0 = 0.0, s1 = 0.0, s2 = 0.0;
            for (int m = 0; m < Q.stages; ++m) {
                const float* cbk = Q.codebooks + (size_t)m * Q.size * 3;
                const int j = rvq_pick(cbk, Q.size, r0, r1, r2);
                Q.idx[(size_t)m * B.total_gauss + g] = (uint8_t)j;
                const float e0 = cbk[3 * j], e1 = cbk[3 * j + 1], e2 = cbk[3 * j + 2];
                r0 = __fsub_rn(r0, e0);
                r1 = __fsub_rn(r1, e1);
                r2 = __fsub_rn(r2, e2);
                s0 = __dadd_rn(s0, (double)e0);
                s1 = __dadd_rn(s1, (double)e1);
                s2 = __dadd_rn(s2, (double)e2);
            }
            cr = (float)s0;
            cg = (float)s1;
            cb = (float)s2;
        }
        int4 r = make_int4(0, 0, 0, 0);
        float4 r0 = make_float4(mx, my, 0.f, 0.f), r1 = make_float4(0.f, cr, cg, cb);
        bool ok = isfinite(mx) && isfinite(my) && isfinite(l1) && isfinite(l2) && isfinite(l3) &&
                  isfinite(cr) && isfinite(cg) && isfinite(cb);
        float ca = 0.f, cbb = 0.f, cc = 0.f, m11 = 0.f, m21 = 0.f, m22 = 0.f;
        if (ok) {
            const float s11 = __fmul_rn(l1, l1);
            const float s12 = __fmul_rn(l1, l2);
            const float s22 = __fadd_rn(__fmul_rn(l2, l2), __fmul_rn(l3, l3));
            const float dd = __fmul_rn(l1, l3);
            const float det = __fmul_rn(dd, dd);
            ok = det != 0.0f;
            if (ok) {
                ca = __fdiv_rn(s22, det);
                cbb = __fdiv_rn(-s12, det);
                cc = __fdiv_rn(s11, det);
                ok = isfinite(det) && isfinite(ca) && isfinite(cbb) && isfinite(cc);
            }
            if (ok) {
                // Scaled inverse Cholesky factor M = sqrt(log2(e)/2) L^-1, so that
                // sigma log2(e) = |M d|^2 (a sum of squares: no cancellation).
                m11 = __fdiv_rn(kSqrtHalfLog2e, l1);
                m22 = __fdiv_rn(kSqrtHalfLog2e, l3);
                m21 = -__fdiv_rn(__fmul_rn(l2, m11), l3);
                ok = isfinite(m11) && isfinite(m21) && isfinite(m22);
            }
            if (ok) {
                const float rx = __fmul_rn(3.0f, fabsf(l1));
                const float ry = __fmul_rn(3.0f, __fsqrt_rn(s22));
                ok = isfinite(rx) && isfinite(ry);
                if (ok) {
                    const float inv_t = 1.0f / (float)B.tile;  // power of two: exact
                    const float ftw = (float)d.tw, fth = (float)d.th;
                    const float fx0 = clampf_(floorf(__fmul_rn(__fsub_rn(mx, rx), inv_t)), 0.0f, ftw);
                    const float fx1 =
                        clampf_(__fadd_rn(floorf(__fmul_rn(__fadd_rn(mx, rx), inv_t)), 1.0f), 0.0f, ftw);
                    const float fy0 = clampf_(floorf(__fmul_rn(__fsub_rn(my, ry), inv_t)), 0.0f, fth);
                    const float fy1 =
                        clampf_(__fadd_rn(floorf(__fmul_rn(__fadd_rn(my, ry), inv_t)), 1.0f), 0.0f, fth);
                    r = make_int4((int)fx0, (int)fy0, (int)fx1, (int)fy1);
                    ok = r.x < r.z && r.y < r.w;
                    if (!ok) r = make_int4(0, 0, 0, 0);
                }
            }
        }
        if (ok) {
            c = (r.z - r.x) * (r.w - r.y);
            r0.z = m11;
            r0.w = m21;
            r1.x = m22;
        }
        rec[2 * (int64_t)g] = r0;
        rec[2 * (int64_t)g + 1] = r1;
        rect[g] = r;
        cnt[g] = c;
        if (M && c > 0) {  // count-matrix rows of the fit path (see bin_cm.cu)
            const int half = threadIdx.x / kCmChunk;
            uint32_t* h = s_h + half * B.total_tiles;
            for (int ty = r.y; ty < r.w; ++ty)
                for (int tx = r.x; tx < r.z; ++tx) atomicAdd(&h[d.tile_base + ty * d.tw + tx], 1u);
            atomicAdd(&s_tot[half], (uint32_t)c);
        }
    }
    const int64_t tot = block_sum<int64_t>((int64_t)c, s_warp);  // its barriers also complete the histograms
    if (threadIdx.x == 0 && blk_sum) blk_sum[blockIdx.x] = tot;
    if (M) {
        const int nchunks = (B.total_gauss + kCmChunk - 1) / kCmChunk;
        for (int q = 0; q < CPB; ++q) {
            const int chunk = CPB * blockIdx.x + q;
            if (chunk >= nchunks) break;
            uint32_t* row = M + (size_t)chunk * B.total_tiles;
            for (int i = threadIdx.x; i < B.total_tiles; i += blockDim.x) row[i] = s_h[q * B.total_tiles + i];
            if (threadIdx.x == 0) chunk_sum[chunk] = s_tot[q];
        }
    }
}

// Block sums of an existing cnt[] (standalone binning), plus zeroing.
__global__ void __launch_bounds__(kProjBlock) k_blocksum(const int32_t* __restrict__ cnt, int32_t n,
                                                         int64_t* __restrict__ blk_sum, ZeroJob zj) {
    __shared__ int64_t s_warp[32];
    pdl_wait();
    zero_job(zj);
    const int g = blockIdx.x * kProjBlock + threadIdx.x;
    const int c = g < n ? cnt[g] : 0;
    const int64_t tot = block_sum<int64_t>((int64_t)c, s_warp);
    if (threadIdx.x == 0) blk_sum[blockIdx.x] = tot;
}

// ---------------------------------------------------------------------------
// Key emission: pair_off = exclusive scan of cnt; the pair j of Gaussian g
// (its rect in row-major order) is (tile, g) at p = pair_off[g] + j (with
// owner: (tile, p) and owner[p] = g), written by the lanes of g's warp in
// turn. Also builds the per-pass digit histograms of the radix sort.
// ---------------------------------------------------------------------------
// Exclusive prefix of block b's pair total over blocks 0 .. b - 1, by a
// look-back that never waits: every block's total is already in blk_sum, and
// a block publishes its inclusive prefix (flag bit 63) as soon as it knows
// it, so a block sums the totals of its nearest predecessors back to the
// first published prefix (32 words per round, warp 0). Integer sums: the
// result does not depend on how far a block had to look.
__device__ int64_t block_prefix_lookback(const int64_t* __restrict__ blk_sum, uint64_t* __restrict__ lb, int b) {
    constexpr uint64_t kPub = 1ull << 63;
    const int lane = threadIdx.x & 31;
    int64_t excl = 0;
    for (int j = b - 1; j >= 0; j -= 32) {
        const int idx = j - lane;  // lane 0 = nearest predecessor
        uint64_t w = 0;
        int64_t v = 0;
        if (idx >= 0) {
            asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(lb + idx) : "memory");
            v = (w & kPub) ? (int64_t)(w & ~kPub) : blk_sum[idx];
        }
        const uint32_t pub = __ballot_sync(0xffffffffu, idx >= 0 && (w & kPub));
        // lanes up to and including the nearest published one
        const uint32_t upto = pub ? ((2u << (__ffs(pub) - 1)) - 1u) : 0xffffffffu;
        excl += warp_sum<int64_t>(((upto >> lane) & 1u) ? v : 0);
        if (pub) break;
    }
    if (lane == 0) {
        const uint64_t w = kPub | (uint64_t)(excl + blk_sum[b]);
        asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(lb + b), "l"(w) : "memory");
    }
    return excl;
}

__global__ void __launch_bounds__(kProjBlock) k_emit(const int4* __restrict__ rect, const int32_t* __restrict__ cnt,
                                                     const int64_t* __restrict__ blk_sum, uint64_t* __restrict__ blk_lb,
                                                     Batch B, int64_t capacity,
                                                     uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                     uint32_t* __restrict__ owner,
                                                     int64_t* __restrict__ pair_off, int64_t* __restrict__ k_dev,
                                                     int64_t* __restrict__ k_max, uint32_t* __restrict__ hist,
                                                     RadixPlan rp, uint32_t* __restrict__ status) {
    __shared__ int64_t s_warp[32];
    __shared__ int64_t s_pre;
    __shared__ uint32_t s_hist[kMaxPasses * kMaxRadix];
    pdl_wait();
    const int n = B.total_gauss;
    for (int i = threadIdx.x; i < kMaxPasses * kMaxRadix; i += blockDim.x) s_hist[i] = 0;
    if (threadIdx.x < 32) {
        const int64_t e = block_prefix_lookback(blk_sum, blk_lb, blockIdx.x);
        if (threadIdx.x == 0) s_pre = e;
    }
    __syncthreads();
    const int64_t pre = s_pre;
    const int g = blockIdx.x * kProjBlock + threadIdx.x;
    const int c = g < n ? cnt[g] : 0;
    const int64_t incl = block_incl_scan<int64_t>((int64_t)c, s_warp);
    const int64_t off = pre + incl - c;
    if (g < n) pair_off[g] = off;
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) {
        const int64_t K = off + c;
        pair_off[n] = K;
        *k_dev = K;
        if (k_max) atomicMax(reinterpret_cast<unsigned long long*>(k_max), (unsigned long long)K);
        if (K > capacity) flag_error(status, kErrCapacity);
    }
    const uint32_t dmask = (1u << rp.dbits) - 1;
    // The warp's Gaussians own one contiguous run of pairs: lane l takes
    // pairs l, l + 32, ... of the run (coalesced stores), finds the owning
    // lane by a search over the warp's count prefix, and the tile from the
    // pair's row-major index j inside the owner's rect.
    {
        const int lane = threadIdx.x & 31;
        int4 r = make_int4(0, 0, 0, 0);
        int tb = 0, tw = 0;
        float inv_w = 0.f;
        if (c > 0) {
            r = rect[g];
            const ImgDesc d = img_desc(B, image_of_gauss(B, g));
            tb = d.tile_base;
            tw = d.tw;
            inv_w = __frcp_rn((float)max(1, r.z - r.x));
        }
        int incl = c;  // warp inclusive prefix of the counts
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        const int woff = incl - c, wtot = __shfl_sync(0xffffffffu, incl, 31);
        const int64_t wbase = __shfl_sync(0xffffffffu, off, 0);  // the run starts at lane 0's offset
        for (int q = lane; q - lane < wtot; q += 32) {  // warp-uniform trip count
            int lo = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int cand = lo + step;
                const int ov = __shfl_sync(0xffffffffu, woff, cand & 31);
                if (cand < 32 && ov <= q) lo = cand;
            }
            const int j = q - __shfl_sync(0xffffffffu, woff, lo);
            const int rx = __shfl_sync(0xffffffffu, r.x, lo), ry = __shfl_sync(0xffffffffu, r.y, lo);
            const int rz = __shfl_sync(0xffffffffu, r.z, lo);
            const int otb = __shfl_sync(0xffffffffu, tb, lo), otw = __shfl_sync(0xffffffffu, tw, lo);
            const float oinv = __shfl_sync(0xffffffffu, inv_w, lo);
            const int64_t pp = wbase + q;
            if (q < wtot && pp < capacity) {
                const int w = max(1, rz - rx);
                // row = j / w: for j < 2^11, (j + 0.5) (1/w) truncated is exact
                // (the product's error stays below 2^-12 / w, less than the
                // 0.5 / w distance of (j + 0.5) / w from an integer)
                const int row = j < 2048 ? __float2int_rz(((float)j + 0.5f) * oinv) : j / w;
                const uint32_t key = (uint32_t)(otb + (ry + row) * otw + rx + (j - row * w));
                keys[pp] = key;
                const uint32_t og = (uint32_t)(blockIdx.x * kProjBlock + (threadIdx.x & ~31) + lo);
                if (owner) {
                    vals[pp] = (uint32_t)pp;  // the sort carries the emission index
                    owner[pp] = og;
                } else {
                    vals[pp] = og;
                }
                for (int ps = 0; ps < rp.passes; ++ps)
                    atomicAdd(&s_hist[ps * kMaxRadix + ((key >> (ps * rp.dbits)) & dmask)], 1u);
            }
        }
    }
    __syncthreads();
    // Flush into one of kHistReplicas copies, spreading the additions of the
    // blocks over more addresses; the sort sums the copies.
    uint32_t* hr = hist + (blockIdx.x % kHistReplicas) * kMaxRadix;
    for (int i = threadIdx.x; i < rp.passes * kMaxRadix; i += blockDim.x) {
        const uint32_t v = s_hist[i];
        if (v) atomicAdd(&hr[(i / kMaxRadix) * kHistReplicas * kMaxRadix + (i % kMaxRadix)], v);
    }
}

// ---------------------------------------------------------------------------
// One stable LSD radix pass (onesweep) over digits of up to 9 bits. Each
// block takes a ticket, ranks its kSortTile keys per digit with warp-level
// multi-split (items ordered by (warp, round, lane) = input order, so the
// ranking is stable), resolves its per-digit global offset with a decoupled
// look-back over lower tickets (bounded spin), and scatters. A thread owns
// digits threadIdx.x and threadIdx.x + kSortThreads in the per-digit phases.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSortThreads) k_onesweep(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, uint32_t* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out, const int64_t* __restrict__ k_dev, int64_t capacity, int shift, int dbits,
    const uint32_t* __restrict__ hist, uint32_t* __restrict__ lookback, uint32_t* __restrict__ ticket,
    uint32_t* __restrict__ status) {
    constexpr int NW = kSortThreads / 32;
    constexpr int DPT = kMaxRadix / kSortThreads;  // digits per thread in the per-digit phases
    __shared__ uint32_t s_wc[NW][kMaxRadix];
    __shared__ uint32_t s_base[kMaxRadix];   // global position of the block's first key of each digit
    __shared__ uint32_t s_boff[kMaxRadix];   // block-local position of the first key of each digit
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_tot0;
    __shared__ uint32_t s_ticket;
    extern __shared__ uint32_t s_stage[];    // [kSortTile] keys, then [kSortTile] values, in digit order
    pdl_wait();
    const int K = (int)min(*k_dev, capacity);
    if (threadIdx.x == 0) s_ticket = atomicAdd(ticket, 1u);
    for (int i = threadIdx.x; i < NW * kMaxRadix; i += kSortThreads) (&s_wc[0][0])[i] = 0;
    __syncthreads();
    const int blk = (int)s_ticket;
    const int64_t start = (int64_t)blk * kSortTile;
    if (start >= K) return;
    const int radix = 1 << dbits;
    const uint32_t mask = (uint32_t)radix - 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    uint32_t key[kSortItems], val[kSortItems], lrank[kSortItems];
    uint32_t dig[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t idx = start + warp * 32 * kSortItems + r * 32 + lane;
        if (idx < K) {
            key[r] = keys_in[idx];
            val[r] = vals_in[idx];
            dig[r] = (key[r] >> shift) & mask;
        } else {
            key[r] = 0;
            val[r] = 0;
            dig[r] = kMaxRadix;  // no digit: not ranked, not stored
        }
    }
    uint32_t* wc = s_wc[warp];
    const uint32_t ltmask = lanemask_lt();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t dg = dig[r];
        // lanes with the same digit (keys past K carry kMaxRadix, a value no
        // digit has, and are grouped apart): one warp match
        const uint32_t peers = __match_any_sync(0xffffffffu, dg);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (lane == leader && dg < kMaxRadix) {
            base = wc[dg];
            wc[dg] = base + __popc(peers);
        }
        base = __shfl_sync(0xffffffffu, base, leader);
        lrank[r] = base + __popc(peers & ltmask);
        __syncwarp();
    }
    __syncthreads();

    // Per digit: exclusive offsets of the warps, the block's total, published
    // at once (an inclusive prefix for the first block).
    uint32_t tot[DPT];
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        const int d = threadIdx.x + q * kSortThreads;
        tot[q] = 0;
        if (d < radix) {
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const uint32_t v = s_wc[w][d];
                s_wc[w][d] = tot[q];
                tot[q] += v;
            }
            st_relaxed_u32(lookback + (size_t)blk * kMaxRadix + d, (blk == 0 ? kFlagPre : kFlagAgg) | tot[q]);
        }
    }
    // Global digit bases: exclusive scan of this pass's histogram, digits
    // [0, kSortThreads) then [kSortThreads, kMaxRadix).
    uint32_t hex[DPT];
    {
        uint32_t carry = 0, lcarry = 0;
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
            const int d = threadIdx.x + q * kSortThreads;
            uint32_t h = 0;
            if (d < radix) {
#pragma unroll
                for (int rep = 0; rep < kHistReplicas; ++rep) h += hist[rep * kMaxRadix + d];
            }
            const uint32_t incl = block_incl_scan<uint32_t>(h, s_warp);  // ends with a barrier
            hex[q] = carry + incl - h;
            if (threadIdx.x == kSortThreads - 1) s_tot0 = incl;
            __syncthreads();
            carry += s_tot0;
            __syncthreads();
            const uint32_t lincl = block_incl_scan<uint32_t>(tot[q], s_warp);
            if (d < radix) s_boff[d] = lcarry + lincl - tot[q];
            if (threadIdx.x == kSortThreads - 1) s_tot0 = lincl;
            __syncthreads();
            lcarry += s_tot0;
            __syncthreads();
        }
    }
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        const int d = threadIdx.x + q * kSortThreads;
        if (d >= radix) continue;
        uint32_t excl = 0;
        if (blk > 0) {
            // Windowed look-back: kWin predecessor words loaded at once
            // (independent loads), consumed nearest first until an inclusive
            // prefix is found or a word is not published yet.
            int j = blk - 1;
            uint32_t spins = 0;
            bool found = false;
            while (!found && j >= 0) {
                uint32_t v[kWin];
#pragma unroll
                for (int i = 0; i < kWin; ++i)
                    v[i] = (j - i >= 0) ? ld_relaxed_u32(lookback + (size_t)(j - i) * kMaxRadix + d) : kFlagPre;
                int used = 0;
#pragma unroll
                for (int i = 0; i < kWin; ++i) {
                    if (found || used != i) break;
                    const uint32_t f = v[i] & (3u << 30);
                    if (f == 0) break;
                    excl += v[i] & kValMask;
                    used = i + 1;
                    if (f == kFlagPre) found = true;
                }
                j -= used;
                if (used == 0) {
                    if (++spins > kSpinLimit) {
                        flag_error(status, kErrTimeout);
                        break;
                    }
                    if (spins > 16) __nanosleep(64);
                }
            }
            st_relaxed_u32(lookback + (size_t)blk * kMaxRadix + d, kFlagPre | ((excl + tot[q]) & kValMask));
        }
        s_base[d] = hex[q] + excl;
    }
    // Stage the block's keys in digit order, then write each digit's run
    // with consecutive threads (coalesced stores).
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t dg = dig[r];
        if (dg < kMaxRadix) {
            const uint32_t li = s_boff[dg] + s_wc[warp][dg] + lrank[r];
            s_stage[li] = key[r];
            s_stage[kSortTile + li] = val[r];
        }
    }
    __syncthreads();
    const int nvalid = (int)min((int64_t)kSortTile, (int64_t)K - start);
    for (int i = threadIdx.x; i < nvalid; i += kSortThreads) {
        const uint32_t kk = s_stage[i];
        const uint32_t dg = (kk >> shift) & mask;
        const uint32_t pos = s_base[dg] + ((uint32_t)i - s_boff[dg]);
        if (pos >= (uint32_t)K) {
            flag_error(status, kErrBounds);
            continue;
        }
        keys_out[pos] = kk;
        vals_out[pos] = s_stage[kSortTile + i];
    }
}

// ranges[t] = [first, last + 1) of key t in the sorted keys; with rec_binned,
// also gathers the record of each sorted pair (rec_binned[k] = rec[ids[k]]),
// one pair per thread so the random reads overlap across the whole grid; with
// emit, the emission index of each sorted pair, which the backward stores its
// sums at. With owner, the sort carried each pair's emission index p: then
// ids[k] = owner[p] and emit[k] = p. Without it (the sort carried the
// Gaussian g), the emission index is pair_off[g] + the pair's row-major
// position in g's rectangle.
__global__ void k_ranges(const uint32_t* __restrict__ keys, uint32_t* __restrict__ ids,
                         const uint32_t* __restrict__ owner, const int64_t* __restrict__ k_dev, int64_t capacity,
                         int2* __restrict__ ranges, Batch B,
                         const float4* __restrict__ rec, float4* __restrict__ rec_binned,
                         const int4* __restrict__ rect, const int64_t* __restrict__ pair_off,
                         uint32_t* __restrict__ emit, uint32_t* __restrict__ status) {
    pdl_wait();
    const int K = (int)min(*k_dev, capacity);
    const int total_tiles = B.total_tiles, n_gauss = B.total_gauss;
    // records moved as one 32-byte access each when both arrays allow it
    const bool v8 = ((reinterpret_cast<uintptr_t>(rec) | reinterpret_cast<uintptr_t>(rec_binned)) & 31) == 0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
        const uint32_t t = keys[k];
        if (owner) {
            // the sorted values are emission indices: the Gaussian is their
            // owner, and the value itself is the pair's emission index
            const uint32_t p = ids[k];
            const uint32_t g = p < (uint32_t)K ? owner[p] : 0xffffffffu;
            if (g < (uint32_t)n_gauss && t < (uint32_t)total_tiles) {
                ids[k] = g;
                if (emit) emit[k] = p;
                if (rec_binned) {
                    if (v8) {
                        float4 a, b;
                        ld_global_v8(rec + 2 * (size_t)g, a, b);
                        st_global_v8(rec_binned + 2 * (size_t)k, a, b);
                    } else {
                        rec_binned[2 * (size_t)k] = rec[2 * (size_t)g];
                        rec_binned[2 * (size_t)k + 1] = rec[2 * (size_t)g + 1];
                    }
                }
            } else {
                flag_error(status, kErrBounds);
            }
        } else if (rec_binned || emit) {
            const uint32_t g = ids[k];
            if (g < (uint32_t)n_gauss && t < (uint32_t)total_tiles) {
                if (rec_binned) {
                    if (v8) {
                        float4 a, b;
                        ld_global_v8(rec + 2 * (size_t)g, a, b);
                        st_global_v8(rec_binned + 2 * (size_t)k, a, b);
                    } else {
                        rec_binned[2 * (size_t)k] = rec[2 * (size_t)g];
                        rec_binned[2 * (size_t)k + 1] = rec[2 * (size_t)g + 1];
                    }
                }
                if (emit) {
                    const ImgDesc d = img_desc(B, image_of_tile(B, (int)t));
                    const int lt = (int)t - d.tile_base;
                    const int4 r = rect[g];
                    const int64_t p = pair_off[g] + (int64_t)(lt / d.tw - r.y) * (r.z - r.x) + (lt % d.tw - r.x);
                    emit[k] = (uint32_t)p;
                }
            } else {
                flag_error(status, kErrBounds);
            }
        }
        if (t >= (uint32_t)total_tiles) continue;
        if (k == 0 || keys[k - 1] != t) ranges[t].x = k;
        if (k == K - 1 || keys[k + 1] != t) ranges[t].y = k + 1;
    }
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

RadixPlan radix_plan(int total_tiles) {
    int bits = 1;
    while (bits < 31 && (int64_t(1) << bits) < (int64_t)total_tiles) ++bits;
    const int passes = (bits + kMaxDigitBits - 1) / kMaxDigitBits;
    const int dbits = (bits + passes - 1) / passes;
    return {bits, passes, dbits};
}

BinWs bin_ws_layout(void* base, int64_t n, int64_t capacity, int total_tiles, bool with_owner) {
    const RadixPlan rp = radix_plan(total_tiles);
    const int64_t nblk = std::max<int64_t>(1, (n + kProjBlock - 1) / kProjBlock);
    const int64_t sblk = std::max<int64_t>(1, (capacity + kSortTile - 1) / kSortTile);
    const int64_t nchunks = std::max<int64_t>(1, (n + kCmChunk - 1) / kCmChunk);
    const int64_t cap = std::max<int64_t>(1, capacity);
    char* b = static_cast<char*>(base);
    size_t off = 0;
    auto take = [&](size_t bytes) -> void* {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return b ? static_cast<void*>(b + o) : nullptr;
    };
    BinWs w{};
    w.cm_path = cm_applies(n, total_tiles);
    w.blk_sum = static_cast<int64_t*>(take(nblk * sizeof(int64_t)));
    if (w.cm_path) {
        w.cm = static_cast<uint32_t*>(take((size_t)nchunks * total_tiles * 4));
        w.chunk_sum = static_cast<uint32_t*>(take((size_t)nchunks * 4));
        w.tile_tot = static_cast<uint32_t*>(take((size_t)total_tiles * 4));
    } else {
        w.keys_tmp = static_cast<uint32_t*>(take(cap * 4));
        w.vals_tmp = static_cast<uint32_t*>(take(cap * 4));
        if (with_owner) w.owner = static_cast<uint32_t*>(take(cap * 4));
    }
    const size_t zero_off = off;
    if (!w.cm_path) {
        w.hist = static_cast<uint32_t*>(take((size_t)rp.passes * kHistReplicas * kMaxRadix * 4));
        w.blk_lb = static_cast<uint64_t*>(take((size_t)nblk * 8));
    }
    if (!w.cm_path) w.lookback = static_cast<uint32_t*>(take((size_t)rp.passes * sblk * kMaxRadix * 4));
    w.tickets = static_cast<uint32_t*>(take(16));
    w.zero = b ? reinterpret_cast<uint32_t*>(b + zero_off) : nullptr;
    w.zero_words = (int64_t)((off - zero_off) / 4);
    w.bytes = off;
    return w;
}

cudaError_t launch_project(const ParamsIn& P, const Batch& B, float4* rec, int4* rect, int32_t* cnt,
                           int64_t* blk_sum, const ZeroJob& zj, cudaStream_t s, uint32_t* cm, uint32_t* chunk_sum) {
    const int nblk = std::max(1, (B.total_gauss + kProjBlock - 1) / kProjBlock);
    const size_t smem = cm ? (size_t)(kProjBlock / kCmChunk) * B.total_tiles * 4 : 0;
    return launch_pdl(k_project, dim3(nblk), dim3(kProjBlock), smem, s, P, B, rec, rect, cnt, blk_sum, zj, cm,
                      chunk_sum);
}

cudaError_t launch_bin(const int4* rect, const int32_t* cnt, const float4* rec, const Batch& B, int64_t capacity,
                       const BinWs& ws, bool blk_sum_ready, uint32_t* keys, uint32_t* ids, int2* ranges,
                       float4* rec_binned, uint32_t* emit, int64_t* pair_off, int64_t* k_dev, int64_t* k_max,
                       uint32_t* status, cudaStream_t s) {
    if (ws.cm_path)
        return launch_bin_cm(rect, cnt, rec, B, capacity, ws, blk_sum_ready, keys, ids, ranges, rec_binned, emit,
                             pair_off, k_dev, k_max, status, s);
    const RadixPlan rp = radix_plan(B.total_tiles);
    const int n = B.total_gauss;
    const int nblk = std::max(1, (n + kProjBlock - 1) / kProjBlock);
    const int64_t sblk = std::max<int64_t>(1, (capacity + kSortTile - 1) / kSortTile);
    if (!blk_sum_ready) {
        ZeroJob zj{};
        zj.p[0] = ws.zero;
        zj.n32[0] = ws.zero_words;
        zj.p[1] = reinterpret_cast<uint32_t*>(ranges);
        zj.n32[1] = (int64_t)B.total_tiles * 2;
        cudaError_t e = launch_pdl(k_blocksum, dim3(nblk), dim3(kProjBlock), 0, s, cnt, n, ws.blk_sum, zj);
        if (e != cudaSuccess) return e;
    }
    uint32_t* ka = (rp.passes & 1) ? ws.keys_tmp : keys;
    uint32_t* va = (rp.passes & 1) ? ws.vals_tmp : ids;
    uint32_t* kb = (rp.passes & 1) ? keys : ws.keys_tmp;
    uint32_t* vb = (rp.passes & 1) ? ids : ws.vals_tmp;
    cudaError_t e = launch_pdl(k_emit, dim3(nblk), dim3(kProjBlock), 0, s, rect, cnt, ws.blk_sum, ws.blk_lb, B,
                               capacity, ka, va, ws.owner, pair_off, k_dev, k_max, ws.hist, rp, status);
    if (e != cudaSuccess) return e;
    // the staging buffer and the static arrays exceed the default 48 KB window
    e = smem_optin(reinterpret_cast<const void*>(k_onesweep), kSortStageBytes);
    if (e != cudaSuccess) return e;
    for (int ps = 0; ps < rp.passes; ++ps) {
        e = launch_pdl(k_onesweep, dim3((unsigned)sblk), dim3(kSortThreads), (size_t)kSortStageBytes, s, ka, va, kb,
                       vb, k_dev, capacity,
                       ps * rp.dbits, rp.dbits, ws.hist + ps * kHistReplicas * kMaxRadix,
                       ws.lookback + (size_t)ps * sblk * kMaxRadix,
                       ws.tickets + ps, status);
        if (e != cudaSuccess) return e;
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    const int rblk = std::max(1, std::min<int>(sm_count() * 8, (int)((capacity + 255) / 256)));
    return launch_pdl(k_ranges, dim3(rblk), dim3(256), 0, s, keys, ids, ws.owner, k_dev, capacity, ranges, B, rec,
                      rec_binned, rect, pair_off, emit, status);
}

}  // namespace gi
