// Tile binning (Sec. 4.1: the spectrum domain is partitioned into tiles that
// are rasterised in parallel).
//
// Output: for every (query q, tile t) the ascending ids n of the Gaussians
// whose footprint rectangle covers t.  This is a stable sort of the keys
// (q, t, n) on the digit (q, t): since keys are produced in ascending n, one
// stable counting-sort pass (a one-digit radix sort with Q*T buckets) puts
// them in (q, t, n) order without ever sorting on n.
//
// Three steps, each bound by memory traffic:
//   1. count   - per (query, chunk of 512 or 1024 Gaussians): smem histogram of the
//                tiles its rectangles cover -> counts[q][t][chunk]
//   2. scan    - exclusive prefix sum over the flattened [q][t][chunk] array
//                (reduce / scan-of-block-sums / down-sweep); the entry of
//                chunk 0 of (q, t) is the CSR offset of that tile list
//   3. scatter - per (query, chunk): stable ranks inside the chunk from
//                warp ballots.  For each warp, colmask[tx] = ballot(lane's
//                rectangle spans column tx) and rowmask[ty] likewise; the
//                lanes covering tile (tx, ty) are colmask & rowmask, so a
//                key's rank inside its warp is popc(mask & lanes_below) and
//                the warps are chained by a per-tile prefix over warps.
#include "kernels.h"

namespace wrf {

namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanBlock = kScanThreads * kScanItems;  // 4096

// Records of query q: n per query at q n, or (multi-scene batches, qbase
// non-NULL) qbase[q+1] - qbase[q] starting at qbase[q].
__device__ __forceinline__ void query_records(const long long *qbase, int n, int q, int &nq,
                                              size_t &base) {
    if (qbase) {
        const long long b0 = qbase[q];
        nq = static_cast<int>(qbase[q + 1] - b0);
        base = static_cast<size_t>(b0);
    } else {
        nq = n;
        base = static_cast<size_t>(q) * n;
    }
}

template <bool WRAP, int CHUNK>
__global__ void __launch_bounds__(256) bin_count_kernel(const float4 *rec, int n, GridView g,
                                                        int C, uint32_t *counts, int *status,
                                                        const long long *qbase) {
    extern __shared__ uint32_t hist[];
    const int c = blockIdx.x, q = blockIdx.y;
    size_t qb;
    query_records(qbase, n, q, n, qb);
    for (int t = threadIdx.x; t < g.T; t += blockDim.x) hist[t] = 0;
    __syncthreads();
    // all of this thread's records are requested before any is used
    constexpr int kPer = CHUNK / 256;
    float4 ra[kPer], rb[kPer];
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int id = c * CHUNK + i * 256 + threadIdx.x;
        if (id < n) {
            const size_t r = qb + id;
            ra[i] = rec[2 * r];
            rb[i] = rec[2 * r + 1];
        }
    }
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int id = c * CHUNK + i * 256 + threadIdx.x;
        if (id >= n) break;
        const float4 a = ra[i], b = rb[i];
        int tx0, tx1, tx2, tx3, ty0, ty1;
        if (!tile_rect_t<WRAP>(a.x, a.y, b.z, b.w, g, tx0, tx1, tx2, tx3, ty0, ty1)) continue;
        // with wrap a tile is rendered with the Gaussian's image nearest to
        // it, which needs every footprint narrower than W - tile width
        if (WRAP && !(__fmul_rn(2.f, b.z) < static_cast<float>(g.W - g.tw)))
            record_status(status, WRF_EUNSUPPORTED);
        for (int ty = ty0; ty <= ty1; ++ty) {
            for (int tx = tx0; tx <= tx1; ++tx) atomicAdd(&hist[ty * g.ntx + tx], 1u);
            if (WRAP)
                for (int tx = tx2; tx <= tx3; ++tx) atomicAdd(&hist[ty * g.ntx + tx], 1u);
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < g.T; t += blockDim.x)
        counts[(static_cast<size_t>(q) * g.T + t) * C + c] = hist[t];
}

// Block-wide exclusive scan of one value per thread (unsigned 64-bit).
__device__ unsigned long long block_exclusive_scan(unsigned long long v,
                                                   unsigned long long *warp_tot,
                                                   unsigned long long *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned long long t = lane < nw ? warp_tot[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    unsigned long long before = w > 0 ? warp_tot[w - 1] : 0ull;
    if (total) *total = warp_tot[nw - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const uint32_t *in,
                                                                   long long M,
                                                                   unsigned long long *sums) {
    __shared__ unsigned long long wt[32];
    long long base = static_cast<long long>(blockIdx.x) * kScanBlock + threadIdx.x * kScanItems;
    unsigned long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < M) s += in[base + i];
    unsigned long long tot;
    block_exclusive_scan(s, wt, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Single block: exclusive scan of the block sums in place; writes the total
// key count and flags overflow.
__global__ void __launch_bounds__(1024) scan_top_kernel(unsigned long long *sums, int nblocks,
                                                        long long cap, long long *n_keys,
                                                        int *status) {
    __shared__ unsigned long long wt[32];
    unsigned long long carry = 0;
    for (int b0 = 0; b0 < nblocks; b0 += 1024) {
        int b = b0 + threadIdx.x;
        unsigned long long v = b < nblocks ? sums[b] : 0ull;
        unsigned long long tot;
        unsigned long long ex = block_exclusive_scan(v, wt, &tot);
        if (b < nblocks) sums[b] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        *n_keys = static_cast<long long>(carry);
        if (carry > static_cast<unsigned long long>(cap) || carry > 0xffffffffull)
            record_status(status, WRF_ENOSPC);
    }
}

__global__ void __launch_bounds__(kScanThreads) scan_down_kernel(
    uint32_t *data, long long M, const unsigned long long *sums, int C, uint32_t *offsets,
    long long QT, const long long *n_keys) {
    __shared__ unsigned long long wt[32];
    long long base = static_cast<long long>(blockIdx.x) * kScanBlock + threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    unsigned long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < M ? data[base + i] : 0u;
        s += v[i];
    }
    unsigned long long run = sums[blockIdx.x] + block_exclusive_scan(s, wt, nullptr);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        long long idx = base + i;
        if (idx < M) {
            uint32_t e = static_cast<uint32_t>(run);
            data[idx] = e;
            if (idx % C == 0) offsets[idx / C] = e;
        }
        run += v[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) offsets[QT] = static_cast<uint32_t>(*n_keys);
}

// CHUNK Gaussians per (query, chunk) CTA, one per thread
template <bool WRAP, int CHUNK>
__global__ void __launch_bounds__(CHUNK, 2048 / CHUNK) bin_scatter_kernel(const float4 *rec, int n, GridView g,
                                                           int C, const uint32_t *excl,
                                                           uint32_t *gids, long long cap,
                                                           const long long *n_keys,
                                                           const long long *qbase) {
    extern __shared__ __align__(16) uint32_t sm[];
    constexpr int kScatterWarps = CHUNK / 32;
    uint32_t *colmask = sm;                                        // [warps][ntx]
    uint32_t *rowmask = colmask + kScatterWarps * g.ntx;           // [warps][nty]
    uint32_t *base = rowmask + kScatterWarps * g.nty;              // [T]
    uint16_t *woff = reinterpret_cast<uint16_t *>(base + g.T);     // [warps][T]
    const int c = blockIdx.x, q = blockIdx.y;
    size_t qb;
    query_records(qbase, n, q, n, qb);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int id = c * CHUNK + threadIdx.x;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
    if (id < n) {
        const size_t r = qb + id;
        a = rec[2 * r];
        b = rec[2 * r + 1];
    }
    // this chunk's start in every tile list of the query, loaded while the
    // records are in flight
    const size_t ebase = static_cast<size_t>(q) * g.T * C + c;
    const uint32_t b0 = threadIdx.x < g.T ? excl[ebase + static_cast<size_t>(threadIdx.x) * C] : 0u;
    int tx0 = 0, tx1 = -1, tx2 = 1, tx3 = 0, ty0 = 0, ty1 = -1;
    const bool valid =
        id < n && tile_rect_t<WRAP>(a.x, a.y, b.z, b.w, g, tx0, tx1, tx2, tx3, ty0, ty1);
    // per warp and tile column / row: the mask of lanes whose rectangle
    // covers it; each lane sets its bit in the few columns and rows it covers
    for (int i = threadIdx.x; i < kScatterWarps * (g.ntx + g.nty); i += blockDim.x) colmask[i] = 0u;
    if (threadIdx.x < g.T) base[threadIdx.x] = b0;
    for (int t = threadIdx.x + blockDim.x; t < g.T; t += blockDim.x)
        base[t] = excl[ebase + static_cast<size_t>(t) * C];
    __syncthreads();
    if (valid) {
        const uint32_t bit = 1u << lane;
        for (int tx = tx0; tx <= tx1; ++tx) atomicOr(&colmask[w * g.ntx + tx], bit);
        if (WRAP)
            for (int tx = tx2; tx <= tx3; ++tx) atomicOr(&colmask[w * g.ntx + tx], bit);
        for (int ty = ty0; ty <= ty1; ++ty) atomicOr(&rowmask[w * g.nty + ty], bit);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < g.T; t += blockDim.x) {
        int tx = t % g.ntx, ty = t / g.ntx;
        uint32_t run = 0;
        for (int ww = 0; ww < kScatterWarps; ++ww) {
            woff[ww * g.T + t] = static_cast<uint16_t>(run);
            run += __popc(colmask[ww * g.ntx + tx] & rowmask[ww * g.nty + ty]);
        }
    }
    __syncthreads();
    if (!valid || *n_keys > cap) return;
    const uint32_t below = (1u << lane) - 1u;
    for (int ty = ty0; ty <= ty1; ++ty) {
        uint32_t rm = rowmask[w * g.nty + ty];
        for (int part = 0; part < (WRAP ? 2 : 1); ++part) {
            const int lo = part == 0 ? tx0 : tx2, hi = part == 0 ? tx1 : tx3;
            for (int tx = lo; tx <= hi; ++tx) {
                int t = ty * g.ntx + tx;
                uint32_t mk = colmask[w * g.ntx + tx] & rm;
                const uint32_t pos = base[t] + woff[w * g.T + t] + __popc(mk & below);
                if (pos < cap) gids[pos] = static_cast<uint32_t>(id);
            }
        }
    }
}

inline size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// Gaussians per binning chunk: 512 for grids of up to 256 tiles (a shorter
// per-tile walk over the chunk's warps, four CTAs per SM), 1024 above (the
// per-(query, tile, chunk) counts, which the scan reads and writes, grow with
// the tile count over the chunk size).
inline int bin_chunk(const GridView &g) { return g.T <= 256 ? 512 : 1024; }

size_t scatter_smem(const GridView &g) {
    const size_t warps = static_cast<size_t>(bin_chunk(g) / 32);
    return warps * (g.ntx + g.nty) * 4 + static_cast<size_t>(g.T) * 4 + warps * g.T * 2;
}

template <int CHUNK>
cudaError_t launch_count_scatter(int phase, const float4 *rec, int n, int Q, const GridView &g,
                                 uint32_t *gids, long long cap, const long long *n_keys,
                                 const BinWs &ws, int *status, const long long *qbase,
                                 cudaStream_t st) {
    dim3 grid(ws.C, Q);
    if (phase == 0) {
        auto kern = g.wrap ? bin_count_kernel<true, CHUNK> : bin_count_kernel<false, CHUNK>;
        kern<<<grid, 256, g.T * 4, st>>>(rec, n, g, ws.C, ws.chunk_counts, status, qbase);
        return cudaGetLastError();
    }
    const size_t smem = scatter_smem(g);
    auto kern = g.wrap ? bin_scatter_kernel<true, CHUNK> : bin_scatter_kernel<false, CHUNK>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<grid, CHUNK, smem, st>>>(rec, n, g, ws.C, ws.chunk_counts, gids, cap, n_keys, qbase);
    return cudaGetLastError();
}

cudaError_t count_scatter(int phase, const float4 *rec, int n, int Q, const GridView &g,
                          uint32_t *gids, long long cap, const long long *n_keys, const BinWs &ws,
                          int *status, const long long *qbase, cudaStream_t st) {
    return bin_chunk(g) == 512
               ? launch_count_scatter<512>(phase, rec, n, Q, g, gids, cap, n_keys, ws, status,
                                           qbase, st)
               : launch_count_scatter<1024>(phase, rec, n, Q, g, gids, cap, n_keys, ws, status,
                                            qbase, st);
}

}  // namespace

size_t bin_ws_layout(int n, int Q, const GridView &g, BinWs *ws, char *base) {
    BinWs w{};
    const int chunk = bin_chunk(g);
    w.C = n > 0 ? (n + chunk - 1) / chunk : 1;
    w.M = static_cast<long long>(Q) * g.T * w.C;
    w.nblocks = static_cast<int>((w.M + kScanBlock - 1) / kScanBlock);
    if (w.nblocks < 1) w.nblocks = 1;
    size_t off = 0;
    w.chunk_counts = reinterpret_cast<uint32_t *>(base ? base + off : nullptr);
    off = align256(off + static_cast<size_t>(w.M) * 4);
    w.block_sums = reinterpret_cast<unsigned long long *>(base ? base + off : nullptr);
    off = align256(off + static_cast<size_t>(w.nblocks) * 8);
    if (ws) *ws = w;
    return off;
}

bool bin_grid_supported(const GridView &g) { return scatter_smem(g) <= 200 * 1024; }

cudaError_t launch_bin(const float4 *rec, int n, int Q, const GridView &g, uint32_t *gids,
                       long long cap, long long *n_keys, uint32_t *offsets, const BinWs &ws,
                       int *status, cudaStream_t st, const long long *qbase) {
    if (Q == 0) return cudaSuccess;
    if (n > 0) {
        cudaError_t e = count_scatter(0, rec, n, Q, g, gids, cap, n_keys, ws, status, qbase, st);
        if (e != cudaSuccess) return e;
    } else {
        cudaError_t e = cudaMemsetAsync(ws.chunk_counts, 0, static_cast<size_t>(ws.M) * 4, st);
        if (e != cudaSuccess) return e;
    }
    scan_reduce_kernel<<<ws.nblocks, kScanThreads, 0, st>>>(ws.chunk_counts, ws.M, ws.block_sums);
    scan_top_kernel<<<1, 1024, 0, st>>>(ws.block_sums, ws.nblocks, cap, n_keys, status);
    scan_down_kernel<<<ws.nblocks, kScanThreads, 0, st>>>(ws.chunk_counts, ws.M, ws.block_sums,
                                                         ws.C, offsets,
                                                         static_cast<long long>(Q) * g.T, n_keys);
    if (n > 0) {
        cudaError_t e = count_scatter(1, rec, n, Q, g, gids, cap, n_keys, ws, status, qbase, st);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace wrf
