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
//   k_count   one block per two chunks: shared-memory tile histograms give
//             the rows of M and the chunk pair totals; clears the binning
//             scratch when asked.
//   k_colscan one block per 16 tiles: column prefix sums over the chunks
//             (P[b][t] = start[t] + sum_{b' < b} M[b'][t], written over M),
//             chained scan of the column totals across tile groups (bounded
//             look-back) -> start, ranges, K and the capacity check.
//   k_place   one block per chunk (two warps per 32 Gaussians): a lane
//             mask per 32 Gaussians of every tile in shared memory gives
//             each pair's rank inside the chunk; the block scatters ids,
//             records and emission indices and writes pair_off.
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
// and returns its count (0 for a bad rect, with *bad set). Threads
// kCmChunk and above of a larger block hold no Gaussian and only take part
// in the scan. Ends with the block scan's barrier.
__device__ __forceinline__ int load_chunk(const int4* __restrict__ rect, const int32_t* __restrict__ cnt,
                                          const Batch& B, int g, ChunkSmem& cs, int* s_warp, bool* bad) {
    const bool holds = threadIdx.x < kCmChunk;
    const bool in = holds && g < B.total_gauss;
    int c = in ? cnt[g] : 0;
    int4 r = in ? rect[g] : make_int4(0, 0, 0, 0);  // issued with the count: no dependent load
    if (c <= 0) r = make_int4(0, 0, 0, 0);
    int2 im = make_int2(0, 0);
    *bad = false;
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
    const int incl = block_incl_scan<int>(c, s_warp);
    if (holds) cs.off[threadIdx.x + 1] = incl;
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
    __shared__ int s_warp[32];
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
// Column scan: block (in ticket order) -> tiles [16 blk, 16 blk + 16); thread
// (tile ti, slab sl) -> chunk rows [sl rs, (sl + 1) rs) of tile ti, 32 slabs.
// Pass 1 sums each slab's rows (kept in registers when they fit). Warp j
// scans tile j's 32 slab partials, giving every slab's offset inside the
// column and the column totals; warp 0 scans the totals over the block's
// tiles and chains the block total through lower tickets (warp-wide
// look-back over 32 predecessors per round, retried until the words up to
// the nearest inclusive prefix are all published; bounded spin). Pass 2
// writes P[r][t] = start[t] + prefix over M in place, and warp w writes the
// sorted keys of the group's tile w (the tile id over its range). The block
// holding the last tile stores K, updates k_max and raises the capacity
// error.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kCmScanThreads) k_colscan(uint32_t* __restrict__ M, int nchunks, int total_tiles,
                                                          int2* __restrict__ ranges, uint32_t* __restrict__ keys,
                                                          int64_t capacity, int64_t* __restrict__ k_dev,
                                                          int64_t* __restrict__ k_max, uint32_t* __restrict__ lookback,
                                                          uint32_t* __restrict__ ticket,
                                                          uint32_t* __restrict__ status) {
    constexpr int TG = kCmGroupTiles, NS = kCmSlabs, NW = kCmScanThreads / 32;
    static_assert(NS == 32 && TG <= NW && 32 % TG == 0, "a warp scans one tile's 32 slabs; one warp per tile");
    __shared__ uint32_t s_part[NS][TG];
    __shared__ uint32_t s_start[TG];
    __shared__ uint32_t s_col[TG];
    __shared__ uint32_t s_ticket;
    pdl_wait();
    if (threadIdx.x == 0) s_ticket = atomicAdd(ticket, 1u);
    __syncthreads();
    const int blk = (int)s_ticket;
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
        if (lane == 31) {
            s_start[warp] = in;  // column total, replaced by the start below
            s_col[warp] = in;
        }
    }
    __syncthreads();
    if (warp == 0) {
        const uint32_t col = lane < TG ? s_start[lane] : 0u;
        uint32_t incl = col;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
        uint32_t excl = 0;
        if (blk == 0) {
            if (lane == 0) st_relaxed_u32(lookback, kFlagPre | (tot & kValMask));
        } else {
            if (lane == 0) st_relaxed_u32(lookback + blk, kFlagAgg | (tot & kValMask));
            int j = blk - 1;
            uint32_t spins = 0;
            while (j >= 0) {
                const int idx = j - lane;  // lane 0 = nearest predecessor
                const uint32_t w = idx >= 0 ? ld_relaxed_u32(lookback + idx) : kFlagPre;
                const uint32_t f = w & (3u << 30);
                const uint32_t pre = __ballot_sync(0xffffffffu, f == kFlagPre);
                const int fp = pre ? __ffs(pre) - 1 : 31;
                const uint32_t upto = fp == 31 ? 0xffffffffu : ((2u << fp) - 1u);  // lanes 0 .. fp
                const uint32_t notready = __ballot_sync(0xffffffffu, f == 0u) & upto;
                if (notready) {
                    if (++spins > kSpinLimit) {
                        if (lane == 0) flag_error(status, kErrTimeout);
                        break;
                    }
                    if (spins > 16) __nanosleep(64);
                    continue;
                }
                excl += warp_sum<uint32_t>(((upto >> lane) & 1u) ? (w & kValMask) : 0u);
                if (pre) break;
                j -= 32;
            }
            if (lane == 0) st_relaxed_u32(lookback + blk, kFlagPre | ((excl + tot) & kValMask));
        }
        const uint32_t start = excl + incl - col;
        if (lane < TG) {
            s_start[lane] = start;
            const int tl = blk * TG + lane;
            if (tl < total_tiles) {
                int2 rg = make_int2(0, 0);
                if (col) {
                    rg.x = (int)min((int64_t)start, capacity);
                    rg.y = (int)min((int64_t)start + col, capacity);
                }
                ranges[tl] = rg;
            }
        }
        if ((blk + 1) * TG >= total_tiles && lane == 0) {
            const int64_t K = (int64_t)excl + tot;
            *k_dev = K;
            if (k_max) atomicMax(reinterpret_cast<unsigned long long*>(k_max), (unsigned long long)K);
            if (K > capacity) flag_error(status, kErrCapacity);
        }
    }
    __syncthreads();
    if (warp < TG) {
        // keys: warp w writes tile (TG blk + w) over its sorted range
        const int tk = blk * TG + warp;
        if (tk < total_tiles) {
            const int64_t s0 = s_start[warp], e0 = min(s0 + (int64_t)s_col[warp], capacity);
            for (int64_t q = s0 + lane; q < e0; q += 32) keys[q] = (uint32_t)tk;
        }
    }
    if (tv && in_regs) {
        uint32_t run = s_start[ti] + s_part[sl][ti];
#pragma unroll
        for (int i = 0; i < kCmRowRegs; ++i) {
            if (r0 + i < r1) M[(size_t)(r0 + i) * total_tiles + t] = run;
            run += v[i];
        }
    } else if (tv) {
        uint32_t run = s_start[ti] + s_part[sl][ti];
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
// group's pairs alternate between them in rounds of 32). Lane masks
// s_m[k][t] (bit l set when local Gaussian 32 k + l covers tile t) are built
// with atomicOr, which is order-independent; then pair (t, g),
// g = 128 b + 32 k + l, lands at
//   P[b][t] + sum_{k' < k} popc(s_m[k'][t]) + popc(s_m[k][t] & bits below l),
// i.e. ascending g inside the tile; the block writes ids and records there
// (the keys come from the column scan). The chunk's row of P and its records
// are staged in shared memory. pair_off = exclusive scan of cnt in emission
// order, the chunk base from the chunk totals.
// ---------------------------------------------------------------------------
constexpr int kPlaceThreads = 2 * kCmChunk;

__global__ void __launch_bounds__(kPlaceThreads) k_place(const int4* __restrict__ rect, const int32_t* __restrict__ cnt,
                                                         const float4* __restrict__ rec, Batch B,
                                                         const uint32_t* __restrict__ P,
                                                         const uint32_t* __restrict__ chunk_sum, int nchunks,
                                                         int64_t capacity, uint32_t* __restrict__ ids,
                                                         float4* __restrict__ rec_binned, uint32_t* __restrict__ emit,
                                                         int64_t* __restrict__ pair_off, uint32_t* __restrict__ status) {
    constexpr int NG = kCmChunk / 32;  // lane groups
    constexpr int kRowLoads = (kCmMaxTiles + kPlaceThreads - 1) / kPlaceThreads;
    extern __shared__ uint32_t s_dyn[];  // [NG][total_tiles] lane masks, then [total_tiles] P row
    __shared__ ChunkSmem cs;
    __shared__ float4 s_rec[kCmChunk][2];
    __shared__ int s_warp[32];
    __shared__ int64_t s_warp64[32];
    pdl_wait();
    const int Tn = B.total_tiles;
    uint32_t* s_m = s_dyn;
    uint32_t* s_p = s_dyn + NG * Tn;
    const int b = blockIdx.x;
    const bool holds = threadIdx.x < kCmChunk;  // threads holding a Gaussian of the chunk
    const int g = b * kCmChunk + threadIdx.x;
    // Independent loads first: the chunk's row of P, the chunk totals below
    // b and this Gaussian's record.
    const uint32_t* prow = P + (size_t)b * Tn;
#pragma unroll
    for (int i = 0; i < kRowLoads; ++i) {
        const int idx = threadIdx.x + i * kPlaceThreads;
        if (idx < Tn) s_p[idx] = prow[idx];
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
    bool bad;
    const int c = load_chunk(rect, cnt, B, g, cs, s_warp, &bad);
    if (bad) flag_error(status, kErrBounds);
    pre = block_sum<int64_t>(pre, s_warp64);
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
    for (int p = p0 + lane; p - lane < wtot; p += 64) {  // warp-uniform trip count
        const int l = warp_owner(woff, p);
        const int j = p - __shfl_sync(0xffffffffu, woff, l);
        if (p < wtot) atomicOr(&s_m[grp * Tn + pair_tile(cs, w0 + l, j)], 1u << l);
    }
    __syncthreads();
    for (int p = p0 + lane; p - lane < wtot; p += 64) {
        const int l = warp_owner(woff, p);
        const int j = p - __shfl_sync(0xffffffffu, woff, l);
        if (p >= wtot) continue;
        const int t = pair_tile(cs, w0 + l, j);
        uint32_t pos = s_p[t] + __popc(s_m[grp * Tn + t] & ((1u << l) - 1u));
        for (int v = 0; v < grp; ++v) pos += __popc(s_m[v * Tn + t]);
        if ((int64_t)pos >= capacity) continue;  // dropped; the scan raised the capacity error
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
    e = launch_pdl(k_colscan, dim3(groups), dim3(kCmScanThreads), 0, s, ws.cm, nchunks, Tn, ranges, keys, capacity,
                   k_dev, k_max, ws.lookback, ws.tickets, status);
    if (e != cudaSuccess) return e;
    // up to 40 KB dynamic + the static layout: above the default 48 KB window
    e = smem_optin(reinterpret_cast<const void*>(k_place), (kCmChunk / 32 + 1) * kCmMaxTiles * 4);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_place, dim3(nchunks), dim3(kPlaceThreads), (size_t)(kCmChunk / 32 + 1) * Tn * 4, s, rect, cnt, rec,
                      B, ws.cm, ws.chunk_sum, nchunks, capacity, ids, rec_binned, emit, pair_off, status);
}

}  // namespace gi
