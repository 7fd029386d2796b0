// bin_cm.cu -- tile binning as a stable counting sort over a count matrix,
// used when the batch has few tiles (cm_applies).
//
// The Gaussians are cut into chunks of kCmChunk consecutive indices. With
// M[b][t] = number of Gaussians of chunk b whose rect covers tile t, the
// sorted position of the pair (t, g), g in chunk b, is
//   start[t] + sum_{b' < b} M[b'][t] + #{g' in chunk b : g' < g, t in rect(g')}
// with start = exclusive scan of the column sums over tiles. This is the
// order the LSD radix path produces (tiles ascending, Gaussian index
// ascending inside a tile), obtained without a sort:
//   k_count   one block per chunk: shared-memory tile histograms give the
//             rows of M and the chunk pair totals; clears the binning
//             scratch when asked.
//   k_colscan one block per 16 tiles: column prefix sums over the chunks
//             (P[b][t] = sum_{b' < b} M[b'][t], written over M) and the
//             column totals tot[t]; no block waits on another.
//   k_place   one block per chunk (two warps per 32 Gaussians): every block
//             scans the column totals itself (start = exclusive scan of tot
//             over the at most kCmMaxTiles tiles); a lane mask per 32
//             Gaussians of every tile in shared memory gives each pair's
//             rank inside the chunk; the block scatters ids, records and
//             emission indices and writes pair_off; the blocks share out
//             the ranges, the keys (the tile id over each range), K and the
//             capacity check.
#include <algorithm>

#include "kernels.cuh"

namespace gi {

namespace {

constexpr int kCmSlabs = 32;                   // k_colscan: row slabs per tile (one warp scans them)
constexpr int kCmScanThreads = kCmGroupTiles * kCmSlabs;  // k_colscan: one thread per (tile, slab)
constexpr int kCmRowRegs = 24;                 // k_colscan: rows a lane keeps in registers between passes

__device__ __forceinline__ void zero_words(uint32_t* p, int64_t n) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < n; i += nth) p[i] = 0u;
}

// True when rect r is a valid tile rectangle of image d holding c tiles.
__device__ __forceinline__ bool rect_ok(const int4& r, const ImgDesc& d, int c) {
    return r.x >= 0 && r.y >= 0 && r.z <= d.tw && r.w <= d.th && r.x < r.z && r.y < r.w &&
           (r.z - r.x) * (r.w - r.y) == c;
}

// Chunk layout shared by k_count and k_place: per Gaussian of the chunk its
// rect, image tile base and tile-row width, and the exclusive prefix of the
// pair counts (off[0..kCmChunk], emission order inside the chunk).
struct ChunkSmem {
    int off[kCmChunk + 1];
    int4 rect[kCmChunk];
    int2 img[kCmChunk];      // (tile_base, tw)
    float inv_w[kCmChunk];  // 1 / rect width, correctly rounded
};

// Pairs are spread over the lanes of the warp that owns their Gaussians:
// pair p of the warp's list (emission order) goes to lane p mod 32, which
// finds the owning lane l (the last lane with woff[l] <= p, woff = the
// warp's exclusive prefix of the counts, one value per lane) by a 5-step
// shuffle search, then the tile from the pair's index j inside the rect.
// The row q = floor(j / w) is computed as (j + 0.5) * (1/w) truncated: with
// j < 2^11 the product's error stays below 2^-12 / w, less than the 0.5 / w
// distance of (j + 0.5) / w from an integer, so q is exact.
__device__ __forceinline__ int warp_owner(int woff, int p) {
    int lo = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const int cand = lo + step;
        const int o = __shfl_sync(0xffffffffu, woff, cand & 31);
        if (cand < 32 && o <= p) lo = cand;
    }
    return lo;
}

__device__ __forceinline__ int pair_tile(const ChunkSmem& cs, int li, int j) {
    const int4 r = cs.rect[li];
    const int w = r.z - r.x;
    const int q = __float2int_rz(((float)j + 0.5f) * cs.inv_w[li]);
    return cs.img[li].x + (r.y + q) * cs.img[li].y + r.x + (j - q * w);
}

// Loads this thread's Gaussian (count, rect, image) into the chunk layout
// and returns its count (0 for a bad rect or a negative count, with *bad
// set). Threads kCmChunk and above of a larger block hold no Gaussian and
// only take part in the scan. The block scan carries a second sum in its
// upper 32 bits: `hi` in, its inclusive block prefix out in *hi_incl. Ends
// with the block scan's barrier.
__device__ __forceinline__ int load_chunk(const int4* __restrict__ rect, const int32_t* __restrict__ cnt,
                                          const Batch& B, int g, ChunkSmem& cs, uint64_t* s_warp, bool* bad,
                                          uint32_t hi = 0u, uint32_t* hi_incl = nullptr) {
    const bool holds = threadIdx.x < kCmChunk;
    const bool in = holds && g < B.total_gauss;
    int c = in ? cnt[g] : 0;
    int4 r = in ? rect[g] : make_int4(0, 0, 0, 0);  // issued with the count: no dependent load
    if (c <= 0) r = make_int4(0, 0, 0, 0);
    int2 im = make_int2(0, 0);
    *bad = c < 0;
    if (c < 0) c = 0;
    if (c > 0) {
        const ImgDesc d = img_desc(B, image_of_gauss(B, g));
        if (rect_ok(r, d, c)) {
            im = make_int2(d.tile_base, d.tw);
        } else {
            *bad = c != 0;
            c = 0;
        }
    }
    if (holds) {
        cs.rect[threadIdx.x] = r;
        cs.img[threadIdx.x] = im;
        cs.inv_w[threadIdx.x] = c > 0 ? __frcp_rn((float)(r.z - r.x)) : 0.f;
    }
    const uint64_t incl = block_incl_scan<uint64_t>(((uint64_t)hi << 32) | (uint32_t)c, s_warp);
    if (holds) cs.off[threadIdx.x + 1] = (int)(uint32_t)incl;
    if (hi_incl) *hi_incl = (uint32_t)(incl >> 32);
    if (threadIdx.x == 0) cs.off[0] = 0;
    __syncthreads();
    return c;
}

// ---------------------------------------------------------------------------
// Count: block = chunk b (kCmChunk threads, one Gaussian each). Every pair
// adds one to the chunk's shared tile histogram, which is written as row b
// of M (all tiles, zeros included); chunk_sum[b] = the chunk's pair count.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kCmChunk) k_count(const int4* __restrict__ rect, const int32_t* __restrict__ cnt,
                                                    Batch B, uint32_t* __restrict__ M,
                                                    uint32_t* __restrict__ chunk_sum, uint32_t* __restrict__ zero,
                                                    int64_t zero_n) {
    extern __shared__ uint32_t s_h[];  // [total_tiles]
    __shared__ ChunkSmem cs;
    __shared__ uint64_t s_warp[32];
    pdl_wait();
    if (zero) zero_words(zero, zero_n);
    const int Tn = B.total_tiles;
    const int b = blockIdx.x;
    for (int i = threadIdx.x; i < Tn; i += blockDim.x) s_h[i] = 0u;
    bool bad;
    const int c = load_chunk(rect, cnt, B, b * kCmChunk + threadIdx.x, cs, s_warp, &bad);  // k_place raises the error
    const int total = cs.off[kCmChunk];
    {
        const int lane = threadIdx.x & 31, w0 = threadIdx.x & ~31;
        const int woff = cs.off[threadIdx.x] - cs.off[w0];
        const int wtot = cs.off[w0 + 32] - cs.off[w0];
        for (int p = lane; p - lane < wtot; p += 32) {  // warp-uniform trip count
            const int l = warp_owner(woff, p);
            const int j = p - __shfl_sync(0xffffffffu, woff, l);
            if (p < wtot) atomicAdd(&s_h[pair_tile(cs, w0 + l, j)], 1u);
        }
    }
    __syncthreads();
    uint32_t* row = M + (size_t)b * Tn;
    for (int i = threadIdx.x; i < Tn; i += blockDim.x) row[i] = s_h[i];
    if (threadIdx.x == 0) chunk_sum[b] = (uint32_t)total;
}

// ---------------------------------------------------------------------------
// Column scan: block blk -> tiles [16 blk, 16 blk + 16); thread (tile ti,
// slab sl) -> chunk rows [sl rs, (sl + 1) rs) of tile ti, 32 slabs. Pass 1
// sums each slab's rows (kept in registers when they fit). Warp j scans tile
// j's 32 slab partials, giving every slab's offset inside the column and the
// column total, which it stores in tot. Pass 2 writes
// P[r][t] = sum_{r' < r} M[r'][t] in place. No block waits on another: the
// start of each tile is added by the placement kernel.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kCmScanThreads) k_colscan(uint32_t* __restrict__ M, int nchunks, int total_tiles,
                                                          uint32_t* __restrict__ tot) {
    constexpr int TG = kCmGroupTiles, NS = kCmSlabs, NW = kCmScanThreads / 32;
    static_assert(NS == 32 && TG <= NW && 32 % TG == 0, "a warp scans one tile's 32 slabs; one warp per tile");
    __shared__ uint32_t s_part[NS][TG];
    pdl_wait();
    const int blk = (int)blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // thread -> (tile ti of the group, row slab sl): TG consecutive tiles of one
    // slab row are one contiguous 4 TG-byte segment of M
    const int ti = threadIdx.x % TG, sl = threadIdx.x / TG;
    const int t = blk * TG + ti;
    const bool tv = t < total_tiles;
    const int rs = (nchunks + NS - 1) / NS;
    const int r0 = min(nchunks, sl * rs), r1 = min(nchunks, r0 + rs);
    const bool in_regs = rs <= kCmRowRegs;  // block-uniform
    uint32_t sum = 0;
    uint32_t v[kCmRowRegs];
    if (tv) {
        if (in_regs) {
#pragma unroll
            for (int i = 0; i < kCmRowRegs; ++i) v[i] = r0 + i < r1 ? M[(size_t)(r0 + i) * total_tiles + t] : 0u;
#pragma unroll
            for (int i = 0; i < kCmRowRegs; ++i) sum += v[i];
        } else {
            int r = r0;
            for (; r + 8 <= r1; r += 8) {
                uint32_t u[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) u[i] = M[(size_t)(r + i) * total_tiles + t];
#pragma unroll
                for (int i = 0; i < 8; ++i) sum += u[i];
            }
            for (; r < r1; ++r) sum += M[(size_t)r * total_tiles + t];
        }
    }
    s_part[sl][ti] = sum;
    __syncthreads();
    if (warp < TG) {
        // warp j scans tile j's slab partials (lane = slab) in place
        const uint32_t x = s_part[lane][warp];
        uint32_t in = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, in, o);
            if (lane >= o) in += u;
        }
        s_part[lane][warp] = in - x;
        if (lane == 31 && blk * TG + warp < total_tiles) tot[blk * TG + warp] = in;
    }
    __syncthreads();
    if (tv && in_regs) {
        uint32_t run = s_part[sl][ti];
#pragma unroll
        for (int i = 0; i < kCmRowRegs; ++i) {
            if (r0 + i < r1) M[(size_t)(r0 + i) * total_tiles + t] = run;
            run += v[i];
        }
    } else if (tv) {
        uint32_t run = s_part[sl][ti];
        int r = r0;
        for (; r + 8 <= r1; r += 8) {
            uint32_t u[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) u[i] = M[(size_t)(r + i) * total_tiles + t];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                M[(size_t)(r + i) * total_tiles + t] = run;
                run += u[i];
            }
        }
        for (; r < r1; ++r) {
            const uint32_t u = M[(size_t)r * total_tiles + t];
            M[(size_t)r * total_tiles + t] = run;
            run += u;
        }
    }
}

// ---------------------------------------------------------------------------
// Place: block = chunk b, two warps per lane group of 32 Gaussians (the
// group's pairs alternate between them in rounds of 32). Every block first
// forms start[t] = sum_{t' < t} tot[t'] (thread i holds tiles
// [kTilesPerThread i, kTilesPerThread (i + 1)), one block scan) and adds it
// to its chunk's row of P. Lane masks s_m[k][t] (bit l set when local
// Gaussian 32 k + l covers tile t) are built with atomicOr, which is
// order-independent; then pair (t, g), g = 128 b + 32 k + l, lands at
//   start[t] + P[b][t] + sum_{k' < k} popc(s_m[k'][t]) + popc(s_m[k][t] & bits below l),
// i.e. ascending g inside the tile; the block writes ids, records and
// emission indices there. pair_off = exclusive scan of cnt in emission
// order, the chunk base from the chunk totals. The blocks share out the
// tile ranges (a thread per tile over the grid), the keys (a warp per tile
// over the grid: the tile id over its range) and, in block 0, K, k_max and
// the capacity check.
// ---------------------------------------------------------------------------
constexpr int kPlaceThreads = 2 * kCmChunk;
constexpr int kTilesPerThread = kCmMaxTiles / kPlaceThreads;
constexpr int kPlaceSmemWords = kCmChunk / 32 + 2;  // per tile: lane masks, P row, start
static_assert(kCmMaxTiles % (4 * kPlaceThreads) == 0, "whole uint4 loads of the tile totals per thread");

__global__ void __launch_bounds__(kPlaceThreads) k_place(const int4* __restrict__ rect, const int32_t* __restrict__ cnt,
                                                         const float4* __restrict__ rec, Batch B,
                                                         const uint32_t* __restrict__ P,
                                                         const uint32_t* __restrict__ tot,
                                                         const uint32_t* __restrict__ chunk_sum, int nchunks,
                                                         int64_t capacity, uint32_t* __restrict__ keys,
                                                         uint32_t* __restrict__ ids, int2* __restrict__ ranges,
                                                         float4* __restrict__ rec_binned, uint32_t* __restrict__ emit,
                                                         int64_t* __restrict__ pair_off, int64_t* __restrict__ k_dev,
                                                         int64_t* __restrict__ k_max, uint32_t* __restrict__ status) {
    constexpr int NG = kCmChunk / 32;  // lane groups
    constexpr int kRowLoads = (kCmMaxTiles + kPlaceThreads - 1) / kPlaceThreads;
    // [NG][total_tiles] lane masks, [total_tiles] P row (+ start), [total_tiles + 1] start
    extern __shared__ uint32_t s_dyn[];
    __shared__ ChunkSmem cs;
    __shared__ float4 s_rec[kCmChunk][2];
    __shared__ uint64_t s_warp[32];
    __shared__ int64_t s_warp64[32];
    pdl_wait();
    const int Tn = B.total_tiles;
    uint32_t* s_m = s_dyn;
    uint32_t* s_p = s_dyn + NG * Tn;
    uint32_t* s_start = s_p + Tn;
    const int b = blockIdx.x;
    const bool holds = threadIdx.x < kCmChunk;  // threads holding a Gaussian of the chunk
    const int g = b * kCmChunk + threadIdx.x;
    // Independent loads first: the chunk's row of P, this thread's tile
    // totals, the chunk totals below b and this Gaussian's record.
    const uint32_t* prow = P + (size_t)b * Tn;
#pragma unroll
    for (int i = 0; i < kRowLoads; ++i) {
        const int idx = threadIdx.x + i * kPlaceThreads;
        if (idx < Tn) s_p[idx] = prow[idx];
    }
    const int t0 = threadIdx.x * kTilesPerThread;
    uint32_t tt[kTilesPerThread];
#pragma unroll
    for (int i = 0; i < kTilesPerThread; i += 4) {
        if (t0 + i + 3 < Tn) {
            const uint4 q = *reinterpret_cast<const uint4*>(tot + t0 + i);
            tt[i] = q.x;
            tt[i + 1] = q.y;
            tt[i + 2] = q.z;
            tt[i + 3] = q.w;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) tt[i + e] = t0 + i + e < Tn ? tot[t0 + i + e] : 0u;
        }
    }
    int64_t pre = 0;
    for (int i = threadIdx.x; i < b; i += 8 * kPlaceThreads) {  // eight predicated loads in flight per round
        uint32_t u[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) u[q] = i + q * kPlaceThreads < b ? chunk_sum[i + q * kPlaceThreads] : 0u;
#pragma unroll
        for (int q = 0; q < 8; ++q) pre += u[q];
    }
    if (rec_binned && holds && g < B.total_gauss) {
        s_rec[threadIdx.x][0] = rec[2 * (size_t)g];
        s_rec[threadIdx.x][1] = rec[2 * (size_t)g + 1];
    }
    for (int i = threadIdx.x; i < NG * Tn; i += kPlaceThreads) s_m[i] = 0u;
    uint32_t tsum = 0;
#pragma unroll
    for (int i = 0; i < kTilesPerThread; ++i) tsum += tt[i];
    bool bad;
    uint32_t tincl = 0;
    const int c = load_chunk(rect, cnt, B, g, cs, s_warp, &bad, tsum, &tincl);  // also scans the tile totals
    if (bad) flag_error(status, kErrBounds);
    {
        // start of this thread's tiles, added to the chunk's row of P
        uint32_t run = tincl - tsum;
#pragma unroll
        for (int i = 0; i < kTilesPerThread; ++i) {
            if (t0 + i < Tn) {
                s_start[t0 + i] = run;
                s_p[t0 + i] += run;
            }
            run += tt[i];
        }
        if (threadIdx.x == kPlaceThreads - 1) s_start[Tn] = tincl;  // K
    }
    pre = block_sum<int64_t>(pre, s_warp64);  // its barriers also publish the starts
    if (holds) {
        const int off = cs.off[threadIdx.x];
        if (g < B.total_gauss) pair_off[g] = pre + off;
        if (b == nchunks - 1 && threadIdx.x == kCmChunk - 1) pair_off[B.total_gauss] = pre + off + c;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = warp >> 1, p0 = 32 * (warp & 1), w0 = 32 * grp;
    const bool v8 = (reinterpret_cast<uintptr_t>(rec_binned) & 31) == 0;  // one 32-byte store per record
    const int woff = cs.off[w0 + lane] - cs.off[w0];
    const int wtot = cs.off[w0 + 32] - cs.off[w0];
    // Pair p of the lane group (emission order) -> owning lane l, index j in
    // its rect, tile t. The first kCache rounds keep (t, l, j) in registers
    // for the scatter after the barrier; later rounds recompute them.
    constexpr int kCache = 4;
    int ct[kCache], clj[kCache];
    auto locate = [&](int p, int& l, int& j) {
        l = warp_owner(woff, p);
        j = p - __shfl_sync(0xffffffffu, woff, l);
    };
#pragma unroll
    for (int r = 0; r < kCache; ++r) {
        const int p = p0 + lane + 64 * r;
        ct[r] = 0;
        clj[r] = 0;
        if (p - lane < wtot) {  // warp-uniform
            int l, j;
            locate(p, l, j);
            if (p < wtot) {
                const int t = pair_tile(cs, w0 + l, j);
                atomicOr(&s_m[grp * Tn + t], 1u << l);
                ct[r] = t;
                clj[r] = (j << 5) | l;  // j < 2048 tiles
            }
        }
    }
    for (int p = p0 + lane + 64 * kCache; p - lane < wtot; p += 64) {  // warp-uniform trip count
        int l, j;
        locate(p, l, j);
        if (p < wtot) atomicOr(&s_m[grp * Tn + pair_tile(cs, w0 + l, j)], 1u << l);
    }
    __syncthreads();
    auto scatter = [&](int t, int l, int j) {
        uint32_t pos = s_p[t] + __popc(s_m[grp * Tn + t] & ((1u << l) - 1u));
        for (int v = 0; v < grp; ++v) pos += __popc(s_m[v * Tn + t]);
        if ((int64_t)pos >= capacity) return;  // dropped; block 0 raises the capacity error
        ids[pos] = (uint32_t)(b * kCmChunk + w0 + l);
        if (emit) emit[pos] = (uint32_t)(pre + cs.off[w0 + l] + j);
        if (rec_binned) {
            if (v8) {
                st_global_v8(rec_binned + 2 * (size_t)pos, s_rec[w0 + l][0], s_rec[w0 + l][1]);
            } else {
                rec_binned[2 * (size_t)pos] = s_rec[w0 + l][0];
                rec_binned[2 * (size_t)pos + 1] = s_rec[w0 + l][1];
            }
        }
    };
#pragma unroll
    for (int r = 0; r < kCache; ++r)
        if (p0 + lane + 64 * r < wtot) scatter(ct[r], clj[r] & 31, clj[r] >> 5);
    for (int p = p0 + lane + 64 * kCache; p - lane < wtot; p += 64) {
        int l, j;
        locate(p, l, j);
        if (p < wtot) scatter(pair_tile(cs, w0 + l, j), l, j);
    }
    // ranges, keys and K, shared out over the grid
    for (int t = b * kPlaceThreads + threadIdx.x; t < Tn; t += gridDim.x * kPlaceThreads) {
        const uint32_t s0 = s_start[t], s1 = s_start[t + 1];
        int2 rg = make_int2(0, 0);
        if (s1 > s0) {
            rg.x = (int)min((int64_t)s0, capacity);
            rg.y = (int)min((int64_t)s1, capacity);
        }
        ranges[t] = rg;
    }
    for (int t = b * (kPlaceThreads / 32) + warp; t < Tn; t += gridDim.x * (kPlaceThreads / 32)) {
        const int64_t s0 = s_start[t], e0 = min((int64_t)s_start[t + 1], capacity);
        for (int64_t q = s0 + lane; q < e0; q += 32) keys[q] = (uint32_t)t;
    }
    if (b == 0 && threadIdx.x == 0) {
        const int64_t K = s_start[Tn];
        *k_dev = K;
        if (k_max) atomicMax(reinterpret_cast<unsigned long long*>(k_max), (unsigned long long)K);
        if (K > capacity) flag_error(status, kErrCapacity);
    }
}

}  // namespace

bool cm_applies(int64_t n, int total_tiles) {
    const int64_t nchunks = std::max<int64_t>(1, (n + kCmChunk - 1) / kCmChunk);
    return total_tiles >= 1 && total_tiles <= kCmMaxTiles && nchunks * total_tiles <= kCmMaxCells;
}

cudaError_t launch_bin_cm(const int4* rect, const int32_t* cnt, const float4* rec, const Batch& B, int64_t capacity,
                          const BinWs& ws, bool prepared, uint32_t* keys, uint32_t* ids, int2* ranges,
                          float4* rec_binned, uint32_t* emit, int64_t* pair_off, int64_t* k_dev, int64_t* k_max,
                          uint32_t* status, cudaStream_t s) {
    const int n = B.total_gauss;
    const int Tn = B.total_tiles;
    const int nchunks = std::max(1, (n + kCmChunk - 1) / kCmChunk);
    const int groups = (Tn + kCmGroupTiles - 1) / kCmGroupTiles;
    cudaError_t e = cudaSuccess;
    if (!prepared) {
        e = launch_pdl(k_count, dim3(nchunks), dim3(kCmChunk), (size_t)Tn * 4, s, rect, cnt, B, ws.cm, ws.chunk_sum,
                       ws.zero, ws.zero_words);
        if (e != cudaSuccess) return e;
    }
    e = launch_pdl(k_colscan, dim3(groups), dim3(kCmScanThreads), 0, s, ws.cm, nchunks, Tn, ws.tile_tot);
    if (e != cudaSuccess) return e;
    // lane masks, P row and starts: up to 48 KB dynamic + the static layout,
    // above the default 48 KB window
    e = smem_optin(reinterpret_cast<const void*>(k_place), kPlaceSmemWords * kCmMaxTiles * 4 + 4);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_place, dim3(nchunks), dim3(kPlaceThreads), (size_t)(kPlaceSmemWords * Tn + 1) * 4, s, rect,
                      cnt, rec, B, ws.cm, ws.tile_tot, ws.chunk_sum, nchunks, capacity, keys, ids, ranges, rec_binned,
                      emit, pair_off, k_dev, k_max, status);
}

}  // namespace gi
